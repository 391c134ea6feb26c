// halfquad.cu -- the half-quadratic minimiser (the dual optimisation that
// section 5 names as a replacement for the conjugate gradient), multiplicative
// (Geman-Reynolds) form, on the rewritten criterion of section 3.4.
//
// phi(sqrt(u)) is concave in u for the Huber, hyperbolic and quadratic phi,
// so phi(r) is the lower envelope of parabolas w r^2 + psi(w) touching at
// w = phi'(r) / (2 r).  Freezing those weights at the iterate f^k turns J into
// a quadratic that lies above J and touches it at f^k; its minimiser solves
//     A f = D,   A = T + sum_e W_e delta_e^H delta_e,   D = H^H s,
// with W_e = lambda_e phi'(r_e) / (2 r_e), delta_e f = f_q - f_p on the edge
// p -> q of Omega1 and f_p on a pixel of Omega0, and T = H^H H the Toeplitz
// operator.  One outer step = the weights, then n_in linear conjugate-gradient
// steps on A f = D from f^k:
//   outer   W from f; J(f) (one reduction)                 k_hq_outer
//           r = D - T f - P f, p = r, rho = <r, r>          k_hq_residual
//   inner   T p (zero-padded FFT, or H^H H p in direct mode)
//           q = T p + P p; alpha = rho / Re<p, q>           k_hq_apply
//           f += alpha p, res += alpha T p, r -= alpha q;
//           beta = <r, r> / rho, rho = <r, r>               k_hq_step
//           p = r + beta p                                  k_hq_dir
// P x = sum_e W_e delta_e^H delta_e x (an edge p -> q with z = x_q - x_p adds
// W_e z at q and -W_e z at p).  res = T f - D is carried along
// (res += alpha T p), so J needs no extra T apply, and D - T f = -res.
// alpha = 0 when Re<p, q> <= 0 and beta = 0 when rho = 0, as in the oracle.
// Vectors FP32, sums float-float, scalars FP64.
//
// The same kernels run the truncated Newton minimiser (the Newton-like method
// section 5 names): the direction s solves half the Newton system,
//     (T + P_W + P_E) s = D - T f - P_W f   (= -grad J / 2),
// by n_in linear CG steps from s = 0, where P_W is the stencil above with
// W_e = lambda_e b(r_e) / 2 and P_E x = sum_e E_e delta_e^T (z_e Re(conj(z_e)
// delta_e x)) with E_e = lambda_e e(r_e) / 2, z_e = delta_e f: together half
// the penalty's Hessian b I + e z z^T (penalty.cuh, phi_curv_e).  Then the
// three majorize-minimize line-search steps of the PR+ CG path along s, and
// f += t3 s, res += t3 T s:
//   outer   W, E from f; J(f)                               k_hq_outer<true>
//           r = D - T f - P_W f, p = r, s = T s = 0          k_hq_residual<true>
//   inner   T p; q = T p + P_W p + P_E p; alpha             k_hq_apply<true>
//           s += alpha p, T s += alpha T p, r -= alpha q     k_hq_step
//           p = r + beta p                                  k_hq_dir
//   search  q1 = Re<s, 2 res>, q2 = Re<s, T s>, t1           k_nt_ls0
//           t2, t3 (the PR+ CG line-search kernel)          k_line_search
//           f += t3 s, res += t3 T s                        k_nt_update
#include <stdint.h>

#include "cg_device.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace spirec {
namespace {

using cgd::f2axpy;
using cgd::f2sub;
using cgd::redot;

// Weights of the quadratic: Wr[p] of the edge p -> p + 1, Wd[p] of p -> p + N,
// W0[p] of the pixel (zero where there is no edge or the lambda is zero);
// for the Newton minimiser also the rank-one coefficients E of the same edges.
struct HqW {
    float* r;
    float* d;
    float* o;
    float* er;
    float* ed;
    float* eo;
};

// P x at pixel p from the weights and x at p and its four neighbours.
__device__ __forceinline__ float2 penalty_normal_at(const float2* x, HqW W, int p, int N)
{
    const int n = p / N, m = p - n * N;
    const float2 xc = __ldcg(x + p);
    float2 out = make_float2(W.o[p] * xc.x, W.o[p] * xc.y);
    if (m + 1 < N) out = f2axpy(-W.r[p], f2sub(__ldcg(x + p + 1), xc), out);
    if (m > 0) out = f2axpy(W.r[p - 1], f2sub(xc, __ldcg(x + p - 1)), out);
    if (n + 1 < N) out = f2axpy(-W.d[p], f2sub(__ldcg(x + p + N), xc), out);
    if (n > 0) out = f2axpy(W.d[p - N], f2sub(xc, __ldcg(x + p - N)), out);
    return out;
}

// P_E x at pixel p: the rank-one Hessian parts of the edges at p and of the
// pixel, z from f and the differences of x on the same edges.
__device__ __forceinline__ float2 penalty_curv_at(const float2* f, const float2* x, HqW W, int p, int N)
{
    const int n = p / N, m = p - n * N;
    const float2 fc = __ldcg(f + p), xc = __ldcg(x + p);
    float2 out = make_float2(0.f, 0.f);
    out = f2axpy(W.eo[p] * redot(fc, xc), fc, out);
    if (m + 1 < N) {
        const float2 z = f2sub(__ldcg(f + p + 1), fc), w = f2sub(__ldcg(x + p + 1), xc);
        out = f2axpy(-W.er[p] * redot(z, w), z, out);
    }
    if (m > 0) {
        const float2 z = f2sub(fc, __ldcg(f + p - 1)), w = f2sub(xc, __ldcg(x + p - 1));
        out = f2axpy(W.er[p - 1] * redot(z, w), z, out);
    }
    if (n + 1 < N) {
        const float2 z = f2sub(__ldcg(f + p + N), fc), w = f2sub(__ldcg(x + p + N), xc);
        out = f2axpy(-W.ed[p] * redot(z, w), z, out);
    }
    if (n > 0) {
        const float2 z = f2sub(fc, __ldcg(f + p - N)), w = f2sub(xc, __ldcg(x + p - N));
        out = f2axpy(W.ed[p - N] * redot(z, w), z, out);
    }
    return out;
}

// Weights at f and J(f) = ||s||^2 - 2 Re<f, D> + Re<f, T f> + R(f)
// = ||s||^2 - Re<f, D> + Re<f, res> + R(f); with NT
// also the rank-one coefficients E = lambda e(r) / 2 of the Newton system.
template <bool NT>
__global__ void __launch_bounds__(kVecThreads, kVecBlocksPerSm)
k_hq_outer(const float2* f, const float2* res, const float2* __restrict__ D, int N, Reg reg, HqW W, float2* parts,
           unsigned* counter, double* scal, double* Jout)
{
    const int P = N * N;
    float v[3] = {0.f, 0.f, 0.f};  // R, Re<f, D>, Re<f, res>
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        const int n = p / N, m = p - n * N;
        const float2 fc = __ldcg(f + p);
        float wr = 0.f, wd = 0.f, wo = 0.f, er = 0.f, ed = 0.f, eo = 0.f;
        if (reg.lambda1 != 0.f) {
            if (m + 1 < N) {
                const float2 z = f2sub(__ldcg(f + p + 1), fc);
                const float r2 = redot(z, z);
                wr = 0.5f * reg.lambda1 * phi_weight(reg.kind, reg.alpha1, r2);
                if (NT) er = 0.5f * reg.lambda1 * phi_curv_e(reg.kind, reg.alpha1, r2);
                v[0] = fmaf(reg.lambda1, phi_value(reg.kind, reg.alpha1, r2), v[0]);
            }
            if (n + 1 < N) {
                const float2 z = f2sub(__ldcg(f + p + N), fc);
                const float r2 = redot(z, z);
                wd = 0.5f * reg.lambda1 * phi_weight(reg.kind, reg.alpha1, r2);
                if (NT) ed = 0.5f * reg.lambda1 * phi_curv_e(reg.kind, reg.alpha1, r2);
                v[0] = fmaf(reg.lambda1, phi_value(reg.kind, reg.alpha1, r2), v[0]);
            }
        }
        if (reg.lambda0 != 0.f) {
            const float r2 = redot(fc, fc);
            wo = 0.5f * reg.lambda0 * phi_weight(reg.kind, reg.alpha0, r2);
            if (NT) eo = 0.5f * reg.lambda0 * phi_curv_e(reg.kind, reg.alpha0, r2);
            v[0] = fmaf(reg.lambda0, phi_value(reg.kind, reg.alpha0, r2), v[0]);
        }
        W.r[p] = wr;
        W.d[p] = wd;
        W.o[p] = wo;
        if (NT) {
            W.er[p] = er;
            W.ed[p] = ed;
            W.eo[p] = eo;
        }
        v[1] += redot(fc, __ldg(D + p));
        v[2] += redot(fc, __ldcg(res + p));
    }
    FF bt[3];
    block_partial<3>(v, bt);
    store_parts<3>(bt, parts, kMaxParts);
    if (last_block(counter)) {
        FF t[3];
        sum_parts_ff<3>(parts, kMaxParts, gridDim.x, t);
        if (threadIdx.x == 0) {
            const double R = ff_to_double(t[0]);
            const double J = scal[S_SS] - ff_to_double(t[1]) + ff_to_double(t[2]) + R;
            scal[S_J] = J;
            scal[S_R] = R;
            if (Jout) *Jout = J;
            *counter = 0u;
        }
    }
}

// r = D - T f - P f = -res - P f, p = r, rho = <r, r>; with NT also s = T s = 0.
template <bool NT>
__global__ void __launch_bounds__(kVecThreads, kVecBlocksPerSm)
k_hq_residual(const float2* f, const float2* res, HqW W, int N, float2* r,
              float2* pv, float2* sv, float2* Ts, float2* parts, unsigned* counter, double* scal)
{
    const int P = N * N;
    float v[1] = {0.f};
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        const float2 pf = penalty_normal_at(f, W, p, N);
        const float2 rs = __ldcg(res + p);
        const float2 rv = make_float2(-rs.x - pf.x, -rs.y - pf.y);
        r[p] = rv;
        pv[p] = rv;
        if (NT) {
            sv[p] = make_float2(0.f, 0.f);
            Ts[p] = make_float2(0.f, 0.f);
        }
        v[0] += redot(rv, rv);
    }
    FF bt[1];
    block_partial<1>(v, bt);
    store_parts<1>(bt, parts, kMaxParts);
    if (last_block(counter)) {
        FF t[1];
        sum_parts_ff<1>(parts, kMaxParts, gridDim.x, t);
        if (threadIdx.x == 0) {
            scal[S_HQ_RHO] = ff_to_double(t[0]);
            *counter = 0u;
        }
    }
}

// q = T p + P p (with NT + P_E p at the iterate f); alpha = rho / Re<p, q>
// (0 unless Re<p, q> > 0).
template <bool NT>
__global__ void __launch_bounds__(kVecThreads, kVecBlocksPerSm)
k_hq_apply(const float2* pv, const float2* Tp, HqW W, const float2* f, int N, float2* q, float2* parts,
           unsigned* counter, double* scal)
{
    const int P = N * N;
    float v[1] = {0.f};
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        float2 pp = penalty_normal_at(pv, W, p, N);
        if (NT) {
            const float2 pe = penalty_curv_at(f, pv, W, p, N);
            pp = make_float2(pp.x + pe.x, pp.y + pe.y);
        }
        const float2 tp = __ldcg(Tp + p);
        const float2 qv = make_float2(tp.x + pp.x, tp.y + pp.y);
        q[p] = qv;
        v[0] += redot(__ldcg(pv + p), qv);
    }
    FF bt[1];
    block_partial<1>(v, bt);
    store_parts<1>(bt, parts, kMaxParts);
    if (last_block(counter)) {
        FF t[1];
        sum_parts_ff<1>(parts, kMaxParts, gridDim.x, t);
        if (threadIdx.x == 0) {
            const double pq = ff_to_double(t[0]);
            scal[S_HQ_ALPHA] = pq > 0.0 ? scal[S_HQ_RHO] / pq : 0.0;
            *counter = 0u;
        }
    }
}

// f += alpha p, res += alpha T p, r -= alpha q; beta = <r, r> / rho
// (0 when rho = 0), rho = <r, r>.
__global__ void __launch_bounds__(kVecThreads, kVecBlocksPerSm)
k_hq_step(float2* f, float2* res, float2* r, const float2* pv, const float2* Tp, const float2* q, int N,
          float2* parts, unsigned* counter, double* scal)
{
    const float a = (float)scal[S_HQ_ALPHA];
    const int P = N * N;
    float v[1] = {0.f};
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        f[p] = f2axpy(a, __ldcg(pv + p), __ldcg(f + p));
        res[p] = f2axpy(a, __ldcg(Tp + p), __ldcg(res + p));
        const float2 rv = f2axpy(-a, __ldcg(q + p), __ldcg(r + p));
        r[p] = rv;
        v[0] += redot(rv, rv);
    }
    FF bt[1];
    block_partial<1>(v, bt);
    store_parts<1>(bt, parts, kMaxParts);
    if (last_block(counter)) {
        FF t[1];
        sum_parts_ff<1>(parts, kMaxParts, gridDim.x, t);
        if (threadIdx.x == 0) {
            const double rho_new = ff_to_double(t[0]), rho = scal[S_HQ_RHO];
            scal[S_HQ_BETA] = rho > 0.0 ? rho_new / rho : 0.0;
            scal[S_HQ_RHO] = rho_new;
            *counter = 0u;
        }
    }
}

// p = r + beta p.
__global__ void __launch_bounds__(kVecThreads, kVecBlocksPerSm) k_hq_dir(const float2* r, float2* pv, int N, const double* scal)
{
    const float b = (float)scal[S_HQ_BETA];
    const int P = N * N;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x)
        pv[p] = f2axpy(b, __ldcg(pv + p), __ldcg(r + p));
}

// The first line-search step along the Newton direction s: q1 = Re<s, 2 res>
// (res = T f - D), q2 = Re<s, T s> and the penalty terms at t = 0 (KIND: phi fixed at
// compile time), then t1 = -(q1 + num0) / (2 q2 + den0) (0 when the
// curvature is not > 0), the quantities the PR+ CG line-search steps use.
template <int KIND>
__global__ void __launch_bounds__(kVecThreads, kVecBlocksPerSm)
k_nt_ls0(const float2* f, const float2* sv, const float2* Ts, const float2* res, int N,
         Reg reg, float2* parts, unsigned* counter, double* scal)
{
    const int P = N * N;
    float v[4] = {0.f, 0.f, 0.f, 0.f};  // q1, q2, num0, den0
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        const float2 sp = __ldcg(sv + p);
        v[0] += 2.f * redot(sp, __ldcg(res + p));
        v[1] += redot(sp, __ldcg(Ts + p));
        cgd::ls_pixel<KIND>(p, N, f, sv, reg, 0.f, v[2], v[3]);
    }
    FF bt[4];
    block_partial<4>(v, bt);
    store_parts<4>(bt, parts, kMaxParts);
    if (last_block(counter)) {
        FF t[4];
        sum_parts_ff<4>(parts, kMaxParts, gridDim.x, t);
        if (threadIdx.x == 0) {
            const double q1 = ff_to_double(t[0]), q2 = ff_to_double(t[1]);
            const double num0 = ff_to_double(t[2]), den0 = ff_to_double(t[3]);
            scal[S_Q1] = q1;
            scal[S_Q2] = q2;
            scal[S_NUM0] = num0;
            scal[S_DEN0] = den0;
            scal[S_T1] = cgd::ls_next(0.0, q1, q2, num0, den0);
            *counter = 0u;
        }
    }
}

// f += t3 s, res += t3 T s.
__global__ void __launch_bounds__(kVecThreads, kVecBlocksPerSm)
k_nt_update(float2* f, float2* res, const float2* sv, const float2* Ts, int N, const double* scal)
{
    const float t = (float)scal[S_T3];
    const int P = N * N;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        f[p] = f2axpy(t, __ldcg(sv + p), __ldcg(f + p));
        res[p] = f2axpy(t, __ldcg(Ts + p), __ldcg(res + p));
    }
}

float2* slot(spirec_plan p, int s) { return reinterpret_cast<float2*>(p->part) + (size_t)s * kMaxParts; }

HqW weights_of(spirec_plan p)
{
    const size_t P = (size_t)p->N * p->N;
    return HqW{p->hqw, p->hqw + P, p->hqw + 2 * P, p->hqw + 3 * P, p->hqw + 4 * P, p->hqw + 5 * P};
}

template <int KIND>
void nt_ls0_k(spirec_plan p, const float2* sv, const float2* Ts)
{
    k_nt_ls0<KIND><<<vec_blocks(p->N), kVecThreads, 0, p->stream>>>(p->f[0], sv, Ts, p->res, p->N, p->reg,
                                                                    slot(p, P_UPD), p->counters + C_UPD, p->scal);
}

}  // namespace

int launch_hq_objective(spirec_plan p, double* Jout)
{
    if (!p->hqw) {
        set_error("the half-quadratic minimiser needs spirec_set_minimiser first");
        return SPIREC_ESTATE;
    }
    if (p->minimiser == SPIREC_MIN_NEWTON)
        k_hq_outer<true><<<vec_blocks(p->N), kVecThreads, 0, p->stream>>>(
            p->f[0], p->res, p->D, p->N, p->reg, weights_of(p), slot(p, P_UPD), p->counters + C_UPD, p->scal, Jout);
    else
        k_hq_outer<false><<<vec_blocks(p->N), kVecThreads, 0, p->stream>>>(
            p->f[0], p->res, p->D, p->N, p->reg, weights_of(p), slot(p, P_UPD), p->counters + C_UPD, p->scal, Jout);
    SPIREC_CK(cudaGetLastError());
    p->launches += 1;
    return SPIREC_OK;
}

// Outer step k: the iterate is f[0], T f - D in res; r in g, p in dbuf[0], T p in
// Td, q in tmp.  J(f^k) goes to Jdev[k].
int hq_outer_step(spirec_plan p, int k, double* Jdev)
{
    const int N = p->N, blocks = vec_blocks(N);
    const HqW W = weights_of(p);
    float2 *f = p->f[0], *pv = p->dbuf[0];
    int rc;
    if ((rc = launch_hq_objective(p, Jdev ? Jdev + k : nullptr)) != SPIREC_OK) return rc;
    k_hq_residual<false><<<blocks, kVecThreads, 0, p->stream>>>(f, p->res, W, N, p->g, pv, nullptr, nullptr,
                                                                slot(p, P_UPD), p->counters + C_UPD, p->scal);
    SPIREC_CK(cudaGetLastError());
    p->launches += 1;
    for (int j = 0; j < p->hq_inner; ++j) {
        rc = p->mode == SPIREC_MODE_DIRECT ? launch_normal_direct(p, pv, p->Td, false)
                                           : launch_toeplitz(p, pv, p->Td, -1);
        if (rc != SPIREC_OK) return rc;
        k_hq_apply<false><<<blocks, kVecThreads, 0, p->stream>>>(pv, p->Td, W, nullptr, N, p->tmp, slot(p, P_UPD),
                                                                 p->counters + C_UPD, p->scal);
        SPIREC_CK(cudaGetLastError());
        k_hq_step<<<blocks, kVecThreads, 0, p->stream>>>(f, p->res, p->g, pv, p->Td, p->tmp, N, slot(p, P_UPD),
                                                         p->counters + C_UPD, p->scal);
        SPIREC_CK(cudaGetLastError());
        k_hq_dir<<<blocks, kVecThreads, 0, p->stream>>>(p->g, pv, N, p->scal);
        SPIREC_CK(cudaGetLastError());
        p->launches += 3;
    }
    return SPIREC_OK;
}

// Newton outer step k: the iterate is f[0], T f - D in res; r in g, p in dbuf[0],
// T p in Td, q in tmp, the direction s in dbuf[1] and T s in f[1].  J(f^k)
// goes to Jdev[k].
int nt_outer_step(spirec_plan p, int k, double* Jdev)
{
    const int N = p->N, blocks = vec_blocks(N);
    const HqW W = weights_of(p);
    float2 *f = p->f[0], *pv = p->dbuf[0], *sv = p->dbuf[1], *Ts = p->f[1];
    int rc;
    if ((rc = launch_hq_objective(p, Jdev ? Jdev + k : nullptr)) != SPIREC_OK) return rc;
    k_hq_residual<true><<<blocks, kVecThreads, 0, p->stream>>>(f, p->res, W, N, p->g, pv, sv, Ts,
                                                               slot(p, P_UPD), p->counters + C_UPD, p->scal);
    SPIREC_CK(cudaGetLastError());
    p->launches += 1;
    for (int j = 0; j < p->hq_inner; ++j) {
        rc = p->mode == SPIREC_MODE_DIRECT ? launch_normal_direct(p, pv, p->Td, false)
                                           : launch_toeplitz(p, pv, p->Td, -1);
        if (rc != SPIREC_OK) return rc;
        k_hq_apply<true><<<blocks, kVecThreads, 0, p->stream>>>(pv, p->Td, W, f, N, p->tmp, slot(p, P_UPD),
                                                                p->counters + C_UPD, p->scal);
        SPIREC_CK(cudaGetLastError());
        k_hq_step<<<blocks, kVecThreads, 0, p->stream>>>(sv, Ts, p->g, pv, p->Td, p->tmp, N, slot(p, P_UPD),
                                                         p->counters + C_UPD, p->scal);
        SPIREC_CK(cudaGetLastError());
        k_hq_dir<<<blocks, kVecThreads, 0, p->stream>>>(p->g, pv, N, p->scal);
        SPIREC_CK(cudaGetLastError());
        p->launches += 3;
    }
    switch (p->reg.kind) {
    case SPIREC_PHI_HUBER: nt_ls0_k<SPIREC_PHI_HUBER>(p, sv, Ts); break;
    case SPIREC_PHI_HYPERBOLIC: nt_ls0_k<SPIREC_PHI_HYPERBOLIC>(p, sv, Ts); break;
    default: nt_ls0_k<SPIREC_PHI_QUADRATIC>(p, sv, Ts); break;
    }
    SPIREC_CK(cudaGetLastError());
    p->launches += 1;
    if ((rc = launch_line_search(p, f, sv, 1)) != SPIREC_OK) return rc;
    if ((rc = launch_line_search(p, f, sv, 2)) != SPIREC_OK) return rc;
    k_nt_update<<<blocks, kVecThreads, 0, p->stream>>>(f, p->res, sv, Ts, N, p->scal);
    SPIREC_CK(cudaGetLastError());
    p->launches += 1;
    return SPIREC_OK;
}

}  // namespace spirec
