// cg.cu -- line search and Polak-Ribiere update (section 3.3) on the
// rewritten criterion (section 3.4, Eq. NewCritLS):
//
//   J(f)      = ||s||^2 - 2 Re<f, D> + Re<f, T f> + R(f)
//   grad J(f) = 2 (T f - D) + grad R(f)       (dJ/dRe f + i dJ/dIm f)
//   R(f)      = lambda1 sum_edges phi1(|f_q - f_p|) + lambda0 sum_p phi0(|f_p|)
//
// One iteration k is six kernels, all on the device, no host round trip:
//   rows_fwd  d = -g + beta d_old; q1 = Re<d, 2 (Tf - D)>; line-search
//             sums at t = 0; row FFTs of d                         (fft.cu)
//   cols      column FFT * Chat * IFFT                             (fft.cu)
//   rows_inv  row IFFTs -> T d; q2 = Re<d, T d>; t1                (fft.cu)
//   2 x line-search step j -> t_{j+1} = t_j - h'(t_j) / curvature (here)
//   update    f += t3 d, T f += t3 T d, g' = grad J(f), J, beta    (here)
// h(t) = J(f + t d) = J_LS(f) + q1 t + q2 t^2 + R(f + t d); each step
// minimises the half-quadratic majorant of h at t_j:
//   h'(t)  = q1 + 2 q2 t + sum_e lambda b(|z_e + t w_e|) Re(conj(z_e + t w_e) w_e)
//   curv   = 2 q2 + sum_e lambda b(|z_e + t w_e|) |w_e|^2
// with z the differences (or pixels) of f and w those of d.  Vectors are FP32;
// sums go through the float-float reductions of reduce.cuh; the scalars are
// FP64 in device memory.
#include <stdint.h>

#include "internal.cuh"
#include "reduce.cuh"

namespace spirec {

// One pixel per thread where the partial slots allow (one wave on 152 SMs at
// N = 512), grid-stride beyond.
int vec_blocks(int N)
{
    const int64_t P = (int64_t)N * N;
    int64_t b = (P + kVecThreads - 1) / kVecThreads;
    if (b > kMaxParts) b = kMaxParts;
    if (b < 1) b = 1;
    return (int)b;
}

namespace {

__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 f2axpy(float t, float2 d, float2 f)
{
    return make_float2(fmaf(t, d.x, f.x), fmaf(t, d.y, f.y));
}
__device__ __forceinline__ float redot(float2 a, float2 b) { return fmaf(a.x, b.x, a.y * b.y); }

// ||s||^2 -> scal[S_SS]
__global__ void k_sumsq(const float2* __restrict__ s, int64_t L, float2* parts, unsigned* counter,
                        double* scal)
{
    float acc = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = s[i];
        acc += redot(v, v);
    }
    float v[1] = {acc};
    FF bt[1];
    block_partial<1>(v, bt);
    store_parts<1>(bt, parts, kMaxParts);
    if (last_block(counter)) {
        FF t[1];
        sum_parts_ff<1>(parts, kMaxParts, gridDim.x, t);
        if (threadIdx.x == 0) {
            scal[S_SS] = ff_to_double(t[0]);
            *counter = 0u;
        }
    }
}

// Line-search step `step` (1 or 2) at t = t_step over the right/down edges of
// every pixel (Omega1) and the pixels (Omega0); the last block forms
// t_{step+1} = t - (q1 + 2 q2 t + num) / (2 q2 + den).  All loads of a pixel
// are issued before any use (neighbour indices clamped, contributions masked)
// so a thread waits on memory once, not once per edge.
__global__ void __launch_bounds__(kVecThreads)
k_line_search(const float2* __restrict__ f, const float2* __restrict__ d, int N, Reg reg, int step,
              float2* parts, unsigned* counter, double* scal)
{
    const double t = scal[S_T1 + step - 1];
    const float tf = (float)t;
    const int P = N * N;
    float num = 0.f, den = 0.f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        const int n = p / N, m = p - n * N;
        const bool has_r = m + 1 < N, has_d = n + 1 < N;
        const int pr = has_r ? p + 1 : p, pd = has_d ? p + N : p;
        const float2 fp = f[p], dp = d[p], fr = f[pr], dr = d[pr], fd = f[pd], dd = d[pd];
        if (reg.lambda1 != 0.f) {
            {
                const float2 w = f2sub(dr, dp);
                const float2 x = f2axpy(tf, w, f2sub(fr, fp));
                const float b = has_r ? reg.lambda1 * phi_weight(reg.kind, reg.alpha1, redot(x, x)) : 0.f;
                num = fmaf(b, redot(x, w), num);
                den = fmaf(b, redot(w, w), den);
            }
            {
                const float2 w = f2sub(dd, dp);
                const float2 x = f2axpy(tf, w, f2sub(fd, fp));
                const float b = has_d ? reg.lambda1 * phi_weight(reg.kind, reg.alpha1, redot(x, x)) : 0.f;
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
    float v[2] = {num, den};
    FF bt[2];
    block_partial<2>(v, bt);
    store_parts<2>(bt, parts, kMaxParts);
    if (last_block(counter)) {
        FF tot[2];
        sum_parts_ff<2>(parts, kMaxParts, gridDim.x, tot);
        if (threadIdx.x == 0) {
            const double q1 = scal[S_Q1], q2 = scal[S_Q2];
            const double h1 = q1 + 2.0 * q2 * t + ff_to_double(tot[0]);
            const double c = 2.0 * q2 + ff_to_double(tot[1]);
            scal[S_T1 + step] = c > 0.0 ? t - h1 / c : t;
            *counter = 0u;
        }
    }
}

// Gradient and step.  Unless FIRST: f_out = f_in + t3 d, Tf += t3 Td.
// Then g = 2 (Tf - D) + grad R(f_out), and the block sums
//   0 <g,g>, 1 Re<g, g_old>, 2 Re<g, d>, 3 R(f), 4 Re<f, D>, 5 Re<f, Tf>.
// The last block forms J = ||s||^2 - 2 Re<f,D> + Re<f,Tf> + R (-> *Jout),
// beta = max(0, (<g,g> - Re<g,g_old>) / <g_old,g_old>), set to 0 when
// Re<g, -g + beta d> >= 0 (restart), and <g,g> for the next iteration.
// Edge of the gradient stencil: an edge from p to q with z = f_q - f_p adds
// +psi(z) at q and -psi(z) at p, psi(z) = b(|z|) z.
template <bool FIRST>
__global__ void __launch_bounds__(kVecThreads)
k_update(const float2* __restrict__ f_in, float2* __restrict__ f_out, const float2* __restrict__ d,
         float2* __restrict__ Tf, const float2* __restrict__ Td, const float2* __restrict__ D,
         float2* __restrict__ g, int N, Reg reg, float2* parts, unsigned* counter, double* scal,
         double* Jout)
{
    const float t = FIRST ? 0.f : (float)scal[S_T3];
    const int P = N * N;
    float a[kUpdVals];
#pragma unroll
    for (int i = 0; i < kUpdVals; ++i) a[i] = 0.f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        const int n = p / N, m = p - n * N;
        const bool has_u = n > 0, has_l = m > 0, has_d = n + 1 < N, has_r = m + 1 < N;
        const int pu = has_u ? p - N : p, pl = has_l ? p - 1 : p;
        const int pd = has_d ? p + N : p, pr = has_r ? p + 1 : p;
        // every load first
        float2 fc = f_in[p], fu = f_in[pu], fl = f_in[pl], fdn = f_in[pd], fr = f_in[pr];
        float2 tf = Tf[p];
        const float2 dv = D[p];
        float2 dc = make_float2(0.f, 0.f), gold = dc, tdv = dc;
        if (!FIRST) {
            dc = d[p];
            const float2 du = d[pu], dl = d[pl], ddn = d[pd], dr = d[pr];
            tdv = Td[p];
            gold = g[p];
            fc = f2axpy(t, dc, fc);
            fu = f2axpy(t, du, fu);
            fl = f2axpy(t, dl, fl);
            fdn = f2axpy(t, ddn, fdn);
            fr = f2axpy(t, dr, fr);
            tf = f2axpy(t, tdv, tf);
            Tf[p] = tf;
            f_out[p] = fc;
        }
        float2 gp = make_float2(2.f * (tf.x - dv.x), 2.f * (tf.y - dv.y));
        float rv = 0.f;
        if (reg.lambda1 != 0.f) {
            const float l1 = reg.lambda1;
            const float2 zu = f2sub(fc, fu), zl = f2sub(fc, fl), zd = f2sub(fdn, fc), zr = f2sub(fr, fc);
            const float ru = redot(zu, zu), rl = redot(zl, zl), rd = redot(zd, zd), rr = redot(zr, zr);
            const float bu = has_u ? l1 * phi_weight(reg.kind, reg.alpha1, ru) : 0.f;
            const float bl = has_l ? l1 * phi_weight(reg.kind, reg.alpha1, rl) : 0.f;
            const float bd = has_d ? l1 * phi_weight(reg.kind, reg.alpha1, rd) : 0.f;
            const float br = has_r ? l1 * phi_weight(reg.kind, reg.alpha1, rr) : 0.f;
            gp = f2axpy(bu, zu, gp);
            gp = f2axpy(bl, zl, gp);
            gp = f2axpy(-bd, zd, gp);
            gp = f2axpy(-br, zr, gp);
            rv = (has_d ? l1 * phi_value(reg.kind, reg.alpha1, rd) : 0.f) +
                 (has_r ? l1 * phi_value(reg.kind, reg.alpha1, rr) : 0.f);
        }
        if (reg.lambda0 != 0.f) {
            const float r2 = redot(fc, fc);
            gp = f2axpy(reg.lambda0 * phi_weight(reg.kind, reg.alpha0, r2), fc, gp);
            rv = fmaf(reg.lambda0, phi_value(reg.kind, reg.alpha0, r2), rv);
        }
        a[0] += redot(gp, gp);
        if (!FIRST) {
            a[1] += redot(gp, gold);
            a[2] += redot(gp, dc);
        }
        a[3] += rv;
        a[4] += redot(fc, dv);
        a[5] += redot(fc, tf);
        g[p] = gp;
    }
    FF bt[kUpdVals];
    block_partial<kUpdVals>(a, bt);
    store_parts<kUpdVals>(bt, parts, kMaxParts);
    if (last_block(counter)) {
        FF tot[kUpdVals];
        sum_parts_ff<kUpdVals>(parts, kMaxParts, gridDim.x, tot);
        if (threadIdx.x == 0) {
            double s[kUpdVals];
            for (int i = 0; i < kUpdVals; ++i) s[i] = ff_to_double(tot[i]);
            const double J = scal[S_SS] - 2.0 * s[4] + s[5] + s[3];
            double beta = 0.0;
            if (!FIRST) {
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

float2* slot(spirec_plan p, int s) { return reinterpret_cast<float2*>(p->part) + (size_t)s * kMaxParts; }

}  // namespace

int launch_data_norm(spirec_plan p)
{
    int blocks = (int)((p->L + 255) / 256);
    if (blocks > 4 * 152) blocks = 4 * 152;
    k_sumsq<<<blocks, 256, 0, p->stream>>>(p->s, p->L, slot(p, P_MISC), p->counters + C_MISC, p->scal);
    SPIREC_CK(cudaGetLastError());
    p->launches += 1;
    return SPIREC_OK;
}

int launch_line_search(spirec_plan p, const float2* f, const float2* d, int step)
{
    k_line_search<<<vec_blocks(p->N), kVecThreads, 0, p->stream>>>(
        f, d, p->N, p->reg, step, slot(p, P_LS), p->counters + C_LS, p->scal);
    SPIREC_CK(cudaGetLastError());
    p->launches += 1;
    return SPIREC_OK;
}

int launch_update(spirec_plan p, const float2* f_in, float2* f_out, const float2* d, float2* Tf,
                  const float2* Td, float2* g, int first, double* Jout)
{
    if (first)
        k_update<true><<<vec_blocks(p->N), kVecThreads, 0, p->stream>>>(
            f_in, f_out, d, Tf, Td, p->D, g, p->N, p->reg, slot(p, P_UPD), p->counters + C_UPD, p->scal, Jout);
    else
        k_update<false><<<vec_blocks(p->N), kVecThreads, 0, p->stream>>>(
            f_in, f_out, d, Tf, Td, p->D, g, p->N, p->reg, slot(p, P_UPD), p->counters + C_UPD, p->scal, Jout);
    SPIREC_CK(cudaGetLastError());
    p->launches += 1;
    return SPIREC_OK;
}

int cg_iteration(spirec_plan p, int k, double* Jdev)
{
    const int N = p->N;
    const float2* fin = p->f[k & 1];
    float2* fout = p->f[(k + 1) & 1];
    float2* dk = p->dbuf[k & 1];
    int rc;
    CgPass a{};
    a.g = p->g;
    a.d_old = p->dbuf[(k + 1) & 1];
    a.d_new = dk;
    a.f = fin;
    a.Tf = p->Tf;
    a.D = p->D;
    a.reg = p->reg;
    a.parts = slot(p, P_ROWA);
    a.counter = p->counters + C_ROWA;
    a.scal = p->scal;
    if ((rc = launch_rows_fwd(p, nullptr, N, N, N, 1, &a)) != SPIREC_OK) return rc;
    if ((rc = launch_cols(p, N, N)) != SPIREC_OK) return rc;
    CgPass c = a;
    c.parts = slot(p, P_ROWC);
    c.counter = p->counters + C_ROWC;
    if ((rc = launch_rows_inv(p, p->Td, 1, dk, &c, 0)) != SPIREC_OK) return rc;
    for (int j = 1; j <= 2; ++j)
        if ((rc = launch_line_search(p, fin, dk, j)) != SPIREC_OK) return rc;
    return launch_update(p, fin, fout, dk, p->Tf, p->Td, p->g, 0, Jdev ? Jdev + k + 1 : nullptr);
}

}  // namespace spirec
