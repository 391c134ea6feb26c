// cg.cu -- penalty stencil, line search and Polak-Ribiere update (section 3.3)
// on the rewritten criterion (section 3.4, Eq. NewCritLS):
//
//   J(f)      = ||s||^2 - 2 Re<f, D> + Re<f, T f> + R(f)
//   grad J(f) = 2 (T f - D) + grad R(f)       (dJ/dRe f + i dJ/dIm f)
//   R(f)      = lambda1 sum_edges phi1(|f_q - f_p|) + lambda0 sum_p phi0(|f_p|)
//
// One iteration, all on the device, no host synchronisation:
//   Toeplitz T d                     -> q2 = Re<d, T d>          (fft.cu)
//   3 x line-search step j           -> t_{j+1} = t_j - h'(t_j) / curvature
//   update: f += t d, T f += t T d, g' = grad J(f), J, dots -> beta
//   direction: d = -g' + beta d      -> q1 = Re<d, 2 (T f - D)>
// Vectors are FP32; every sum goes through the FP64 block/last-block
// reduction of reduce.cuh; scalars live in FP64 device memory.
#include <stdint.h>

#include "internal.cuh"
#include "reduce.cuh"

namespace spirec {

int vec_blocks(int N)
{
    const int64_t P = (int64_t)N * N;
    int64_t b = (P + kVecThreads - 1) / kVecThreads;
    if (b > 4 * 152) b = 4 * 152;
    if (b < 1) b = 1;
    return (int)b;
}

namespace {

// b(r) = phi'(r) / r from r^2 (the half-quadratic weight).
__device__ __forceinline__ float phi_weight(int kind, float alpha, float r2)
{
    if (kind == SPIREC_PHI_HUBER) return r2 <= alpha * alpha ? 2.f : 2.f * alpha * rsqrtf(r2);
    if (kind == SPIREC_PHI_HYPERBOLIC) return 2.f * alpha * rsqrtf(fmaf(alpha, alpha, r2));
    return 2.f;
}

// phi(r) from r^2.  The hyperbolic form uses sqrt(a^2+r^2)-a = r^2/(sqrt(a^2+r^2)+a).
__device__ __forceinline__ float phi_value(int kind, float alpha, float r2)
{
    if (kind == SPIREC_PHI_HUBER)
        return r2 <= alpha * alpha ? r2 : 2.f * alpha * sqrtf(r2) - alpha * alpha;
    if (kind == SPIREC_PHI_HYPERBOLIC) return 2.f * alpha * r2 / (sqrtf(fmaf(alpha, alpha, r2)) + alpha);
    return r2;
}

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 f2axpy(float t, float2 d, float2 f)
{
    return make_float2(fmaf(t, d.x, f.x), fmaf(t, d.y, f.y));
}
__device__ __forceinline__ float redot(float2 a, float2 b) { return fmaf(a.x, b.x, a.y * b.y); }

// ||s||^2 -> scal[S_SS]
__global__ void k_sumsq(const float2* __restrict__ s, int64_t L, double* part, unsigned* counter,
                        double* scal)
{
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = s[i];
        acc += (double)redot(v, v);
    }
    const double tot = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
    if (last_block(counter)) {
        const double v = sum_parts(part, gridDim.x);
        if (threadIdx.x == 0) {
            scal[S_SS] = v;
            *counter = 0u;
        }
    }
}

// Line-search step `step` (0, 1, 2) at t = t_step (t_0 = 0):
//   num = sum_e lambda b(|z_e + t w_e|) Re(conj(z_e + t w_e) w_e)
//   den = sum_e lambda b(|z_e + t w_e|) |w_e|^2
// over the right/down edges of every pixel (Omega1) and the pixels (Omega0);
// the last block forms t_{step+1} = t - (q1 + 2 q2 t + num) / (2 q2 + den).
__global__ void k_line_search(const float2* __restrict__ f, const float2* __restrict__ d, int N,
                              Reg reg, int step, double* part, unsigned* counter, double* scal)
{
    const double t = step == 0 ? 0.0 : scal[S_T1 + step - 1];
    const float tf = (float)t;
    const int64_t P = (int64_t)N * N;
    float num = 0.f, den = 0.f;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(p / N), m = (int)(p - (int64_t)n * N);
        const float2 fp = f[p], dp = d[p];
        if (reg.lambda1 != 0.f) {
            if (m + 1 < N) {
                const float2 w = f2sub(d[p + 1], dp);
                const float2 x = f2axpy(tf, w, f2sub(f[p + 1], fp));
                const float b = reg.lambda1 * phi_weight(reg.kind, reg.alpha1, redot(x, x));
                num = fmaf(b, redot(x, w), num);
                den = fmaf(b, redot(w, w), den);
            }
            if (n + 1 < N) {
                const float2 w = f2sub(d[p + N], dp);
                const float2 x = f2axpy(tf, w, f2sub(f[p + N], fp));
                const float b = reg.lambda1 * phi_weight(reg.kind, reg.alpha1, redot(x, x));
                num = fmaf(b, redot(x, w), num);
                den = fmaf(b, redot(w, w), den);
            }
        }
        if (reg.lambda0 != 0.f) {
            const float2 x = f2axpy(tf, dp, fp);
            const float b = reg.lambda0 * phi_weight(reg.kind, reg.alpha0, redot(x, x));
            num = fmaf(b, redot(x, dp), num);
            den = fmaf(b, redot(dp, dp), den);
        }
    }
    const double bn = block_sum((double)num);
    const double bd = block_sum((double)den);
    if (threadIdx.x == 0) {
        part[P_LS * kMaxParts + blockIdx.x] = bn;
        part[(P_LS + 1) * kMaxParts + blockIdx.x] = bd;
    }
    if (last_block(counter)) {
        const double sn = sum_parts(part + P_LS * kMaxParts, gridDim.x);
        const double sd = sum_parts(part + (P_LS + 1) * kMaxParts, gridDim.x);
        if (threadIdx.x == 0) {
            const double q1 = scal[S_Q1], q2 = scal[S_Q2];
            const double h1 = q1 + 2.0 * q2 * t + sn;
            const double c = 2.0 * q2 + sd;
            scal[S_T1 + step] = c > 0.0 ? t - h1 / c : t;
            *counter = 0u;
        }
    }
}

// Gradient and step.  With first == 0: f_out = f_in + t3 d, Tf += t3 Td.
// Then g = 2 (Tf - D) + grad R(f_out), and the block sums
//   0 <g,g>, 1 Re<g, g_old>, 2 Re<g, d>, 3 R(f), 4 Re<f, D>, 5 Re<f, Tf>.
// The last block forms J = ||s||^2 - 2 Re<f,D> + Re<f,Tf> + R (-> *Jout),
// beta = max(0, (<g,g> - Re<g,g_old>) / <g_old,g_old>), set to 0 when
// Re<g, -g + beta d> >= 0 (restart), and <g,g> for the next iteration.
__global__ void __launch_bounds__(kVecThreads)
k_update(const float2* __restrict__ f_in, float2* __restrict__ f_out, const float2* __restrict__ d,
         float2* __restrict__ Tf, const float2* __restrict__ Td, const float2* __restrict__ D,
         float2* __restrict__ g, int N, Reg reg, int first, double* part, unsigned* counter,
         double* scal, double* Jout)
{
    const float t = first ? 0.f : (float)scal[S_T3];
    const int64_t P = (int64_t)N * N;
    float a[kUpdVals];
#pragma unroll
    for (int i = 0; i < kUpdVals; ++i) a[i] = 0.f;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(p / N), m = (int)(p - (int64_t)n * N);
        // f at p and its four neighbours after the step
        const float2 fp = first ? f_in[p] : f2axpy(t, d[p], f_in[p]);
        float2 tf = Tf[p];
        if (!first) {
            tf = f2axpy(t, Td[p], tf);
            Tf[p] = tf;
            f_out[p] = fp;
        }
        const float2 dv = D[p];
        float2 gp = make_float2(2.f * (tf.x - dv.x), 2.f * (tf.y - dv.y));
        float rv = 0.f;
        if (reg.lambda1 != 0.f) {
            const float l1 = reg.lambda1;
            // edges into p (from up, left): +psi(f_p - f_q); out of p (down, right): -psi(f_q - f_p)
            if (n > 0) {
                const float2 fq = first ? f_in[p - N] : f2axpy(t, d[p - N], f_in[p - N]);
                const float2 z = f2sub(fp, fq);
                const float b = l1 * phi_weight(reg.kind, reg.alpha1, redot(z, z));
                gp = f2axpy(b, z, gp);
            }
            if (m > 0) {
                const float2 fq = first ? f_in[p - 1] : f2axpy(t, d[p - 1], f_in[p - 1]);
                const float2 z = f2sub(fp, fq);
                const float b = l1 * phi_weight(reg.kind, reg.alpha1, redot(z, z));
                gp = f2axpy(b, z, gp);
            }
            if (n + 1 < N) {
                const float2 fq = first ? f_in[p + N] : f2axpy(t, d[p + N], f_in[p + N]);
                const float2 z = f2sub(fq, fp);
                const float r2 = redot(z, z);
                const float b = l1 * phi_weight(reg.kind, reg.alpha1, r2);
                gp = f2axpy(-b, z, gp);
                rv = fmaf(l1, phi_value(reg.kind, reg.alpha1, r2), rv);
            }
            if (m + 1 < N) {
                const float2 fq = first ? f_in[p + 1] : f2axpy(t, d[p + 1], f_in[p + 1]);
                const float2 z = f2sub(fq, fp);
                const float r2 = redot(z, z);
                const float b = l1 * phi_weight(reg.kind, reg.alpha1, r2);
                gp = f2axpy(-b, z, gp);
                rv = fmaf(l1, phi_value(reg.kind, reg.alpha1, r2), rv);
            }
        }
        if (reg.lambda0 != 0.f) {
            const float r2 = redot(fp, fp);
            const float b = reg.lambda0 * phi_weight(reg.kind, reg.alpha0, r2);
            gp = f2axpy(b, fp, gp);
            rv = fmaf(reg.lambda0, phi_value(reg.kind, reg.alpha0, r2), rv);
        }
        a[0] += redot(gp, gp);
        if (!first) {
            a[1] += redot(gp, g[p]);
            a[2] += redot(gp, d[p]);
        }
        a[3] += rv;
        a[4] += redot(fp, dv);
        a[5] += redot(fp, tf);
        g[p] = gp;
    }
    double tot[kUpdVals];
#pragma unroll
    for (int i = 0; i < kUpdVals; ++i) tot[i] = block_sum((double)a[i]);
    if (threadIdx.x == 0)
        for (int i = 0; i < kUpdVals; ++i) part[(P_UPD + i) * kMaxParts + blockIdx.x] = tot[i];
    if (last_block(counter)) {
        double s[kUpdVals];
        for (int i = 0; i < kUpdVals; ++i) s[i] = sum_parts(part + (P_UPD + i) * kMaxParts, gridDim.x);
        if (threadIdx.x == 0) {
            const double J = scal[S_SS] - 2.0 * s[4] + s[5] + s[3];
            double beta = 0.0;
            if (!first) {
                const double gg_old = scal[S_GG];
                beta = gg_old > 0.0 ? (s[0] - s[1]) / gg_old : 0.0;
                if (beta < 0.0) beta = 0.0;
                if (-s[0] + beta * s[2] >= 0.0) beta = 0.0;
            }
            scal[S_GG] = s[0];
            scal[S_BETA] = beta;
            scal[S_J] = J;
            scal[S_R] = s[3];
            if (Jout) *Jout = J;
            *counter = 0u;
        }
    }
}

// d = -g + beta d (d = -g when beta == 0), and q1 = Re<d, 2 (Tf - D)>.
__global__ void __launch_bounds__(kVecThreads)
k_direction(float2* __restrict__ d, const float2* __restrict__ g, const float2* __restrict__ Tf,
            const float2* __restrict__ D, int N, double* part, unsigned* counter, double* scal)
{
    const double beta_d = scal[S_BETA];
    const float beta = (float)beta_d;
    const int64_t P = (int64_t)N * N;
    float acc = 0.f;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        const float2 gp = g[p];
        float2 dn = make_float2(-gp.x, -gp.y);
        if (beta_d != 0.0) dn = f2axpy(beta, d[p], dn);
        d[p] = dn;
        const float2 tf = Tf[p], dv = D[p];
        acc += 2.f * redot(dn, f2sub(tf, dv));
    }
    const double tot = block_sum((double)acc);
    if (threadIdx.x == 0) part[P_Q1 * kMaxParts + blockIdx.x] = tot;
    if (last_block(counter)) {
        const double v = sum_parts(part + P_Q1 * kMaxParts, gridDim.x);
        if (threadIdx.x == 0) {
            scal[S_Q1] = v;
            *counter = 0u;
        }
    }
}

}  // namespace

int launch_data_norm(spirec_plan p)
{
    int blocks = (int)((p->L + 255) / 256);
    if (blocks > 4 * 152) blocks = 4 * 152;
    k_sumsq<<<blocks, 256, 0, p->stream>>>(p->s, p->L, p->part + P_MISC * kMaxParts,
                                           p->counters + C_MISC, p->scal);
    SPIREC_CK(cudaGetLastError());
    p->launches += 1;
    return SPIREC_OK;
}

int launch_line_search(spirec_plan p, const float2* f, int step)
{
    k_line_search<<<vec_blocks(p->N), kVecThreads, 0, p->stream>>>(
        f, p->d, p->N, p->reg, step, p->part, p->counters + C_LS, p->scal);
    SPIREC_CK(cudaGetLastError());
    p->launches += 1;
    return SPIREC_OK;
}

int launch_update(spirec_plan p, const float2* f_in, float2* f_out, float2* Tf, const float2* Td,
                  float2* g, int first, double* Jout)
{
    k_update<<<vec_blocks(p->N), kVecThreads, 0, p->stream>>>(
        f_in, f_out, p->d, Tf, Td, p->D, g, p->N, p->reg, first, p->part, p->counters + C_UPD,
        p->scal, Jout);
    SPIREC_CK(cudaGetLastError());
    p->launches += 1;
    return SPIREC_OK;
}

int launch_direction(spirec_plan p, int first)
{
    (void)first;
    k_direction<<<vec_blocks(p->N), kVecThreads, 0, p->stream>>>(
        p->d, p->g, p->Tf, p->D, p->N, p->part, p->counters + C_DIR, p->scal);
    SPIREC_CK(cudaGetLastError());
    p->launches += 1;
    return SPIREC_OK;
}

int cg_iteration(spirec_plan p, int k, double* Jdev)
{
    const float2* fin = p->f[k & 1];
    float2* fout = p->f[(k + 1) & 1];
    int rc;
    if ((rc = launch_toeplitz(p, p->d, p->Td, S_Q2)) != SPIREC_OK) return rc;
    for (int j = 0; j < 3; ++j)
        if ((rc = launch_line_search(p, fin, j)) != SPIREC_OK) return rc;
    if ((rc = launch_update(p, fin, fout, p->Tf, p->Td, p->g, 0, Jdev ? Jdev + k + 1 : nullptr)) != SPIREC_OK)
        return rc;
    return launch_direction(p, 0);
}

}  // namespace spirec
