// cg.cu -- line search and Polak-Ribiere update (section 3.3) on the
// rewritten criterion (section 3.4, Eq. NewCritLS):
//
//   J(f)      = ||s||^2 - 2 Re<f, D> + Re<f, T f> + R(f)
//   grad J(f) = 2 (T f - D) + grad R(f)       (dJ/dRe f + i dJ/dIm f)
// The iteration carries res = T f - D, not T f: it starts as T x0 - D and
// moves by t T d with every step.
//   R(f)      = lambda1 sum_edges phi1(|f_q - f_p|) + lambda0 sum_p phi0(|f_p|)
//
// One iteration k is six kernels, all on the device, no host round trip:
//   rows_fwd  d = -g + beta d_old; q1 = Re<d, 2 res>; line-search
//             sums at t = 0; row FFTs of d                         (fft.cu)
//   cols      column FFT * Chat * IFFT                             (fft.cu)
//   rows_inv  row IFFTs -> T d; q2 = Re<d, T d>; t1                (fft.cu)
//   2 x line-search step j -> t_{j+1} = t_j - h'(t_j) / curvature (here)
//   update    f += t3 d, res += t3 T d, g' = grad J(f), J, beta    (here)
// h(t) = J(f + t d) = J_LS(f) + q1 t + q2 t^2 + R(f + t d); each step
// minimises the half-quadratic majorant of h at t_j:
//   h'(t)  = q1 + 2 q2 t + sum_e lambda b(|z_e + t w_e|) Re(conj(z_e + t w_e) w_e)
//   curv   = 2 q2 + sum_e lambda b(|z_e + t w_e|) |w_e|^2
// with z the differences (or pixels) of f and w those of d.  Vectors are FP32;
// sums go through the float-float reductions of reduce.cuh; the scalars are
// FP64 in device memory.
#include <stdint.h>

#include "cg_device.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace spirec {

// One pixel per thread up to kVecBlocksPerSm resident blocks an SM (the
// vector kernels are built to fit that many), grid-stride beyond: a single
// wave, and few block partials for the last block to add.
int vec_blocks(int N)
{
    const int64_t P = (int64_t)N * N;
    int sms = 0;
    if (device_sms(&sms) != SPIREC_OK || sms <= 0) sms = 152;
    int64_t b = (P + kVecThreads - 1) / kVecThreads;
    if (b > (int64_t)kVecBlocksPerSm * sms) b = (int64_t)kVecBlocksPerSm * sms;
    if (b > kMaxParts) b = kMaxParts;
    if (b < 1) b = 1;
    return (int)b;
}

namespace {

using cgd::redot;

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

// Line-search step `step` (1 or 2) at t = t_step; the last block forms
// t_{step+1} (cgd::ls_next).  KIND: phi fixed at compile time.
template <int KIND>
__global__ void __launch_bounds__(kVecThreads, kVecBlocksPerSm)
k_line_search(const float2* f, const float2* d, int N, Reg reg, int step, float2* parts,
              unsigned* counter, double* scal)
{
    const double t = scal[S_T1 + step - 1];
    const float tf = (float)t;
    const int P = N * N;
    float v[2] = {0.f, 0.f};
#pragma unroll 2
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x)
        cgd::ls_pixel<KIND>(p, N, f, d, reg, tf, v[0], v[1]);
    FF bt[2];
    block_partial<2>(v, bt);
    store_parts<2>(bt, parts, kMaxParts);
    if (last_block(counter)) {
        FF tot[2];
        sum_parts_ff<2>(parts, kMaxParts, gridDim.x, tot);
        if (threadIdx.x == 0) {
            scal[S_T1 + step] = cgd::ls_next(t, scal[S_Q1], scal[S_Q2], ff_to_double(tot[0]), ff_to_double(tot[1]));
            *counter = 0u;
        }
    }
}

// Gradient and step (cgd::update_pixel); the last block forms J and beta.
template <bool FIRST, int KIND>
__global__ void __launch_bounds__(kVecThreads, kVecBlocksPerSm)
k_update(const float2* f_in, float2* f_out, const float2* d, float2* res, const float2* Td,
         const float2* __restrict__ D, float2* g, int N, Reg reg, float2* parts, unsigned* counter,
         double* scal, double* Jout)
{
    const float t = FIRST ? 0.f : (float)scal[S_T3];
    const int P = N * N;
    float a[kUpdVals];
#pragma unroll
    for (int i = 0; i < kUpdVals; ++i) a[i] = 0.f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x)
        cgd::update_pixel<FIRST, KIND>(p, N, f_in, f_out, d, res, Td, D, g, reg, t, a);
    FF bt[kUpdVals];
    block_partial<kUpdVals>(a, bt);
    store_parts<kUpdVals>(bt, parts, kMaxParts);
    if (last_block(counter)) {
        FF tot[kUpdVals];
        sum_parts_ff<kUpdVals>(parts, kMaxParts, gridDim.x, tot);
        if (threadIdx.x == 0) {
            double s[kUpdVals];
            for (int i = 0; i < kUpdVals; ++i) s[i] = ff_to_double(tot[i]);
            double J, beta;
            cgd::update_finish(s, scal[S_SS], scal[S_GG], FIRST, &J, &beta);
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

// res = res - D (res holds T x0) or res = -D (x0 = 0): the residual the
// iteration starts from.
__global__ void k_res_init(float2* res, const float2* __restrict__ D, int64_t n, int have_tx)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 dv = D[i];
        const float2 t = have_tx ? res[i] : make_float2(0.f, 0.f);
        res[i] = make_float2(t.x - dv.x, t.y - dv.y);
    }
}

}  // namespace

int launch_res_init(spirec_plan p, float2* res, bool have_tx)
{
    k_res_init<<<vec_blocks(p->N), kVecThreads, 0, p->stream>>>(res, p->D, (int64_t)p->N * p->N, have_tx ? 1 : 0);
    SPIREC_CK(cudaGetLastError());
    p->launches += 1;
    return SPIREC_OK;
}

int launch_data_norm(spirec_plan p)
{
    int blocks = (int)((p->L + 255) / 256);
    if (blocks > 4 * 152) blocks = 4 * 152;
    k_sumsq<<<blocks, 256, 0, p->stream>>>(p->s, p->L, slot(p, P_MISC), p->counters + C_MISC, p->scal);
    SPIREC_CK(cudaGetLastError());
    p->launches += 1;
    return SPIREC_OK;
}

namespace {
template <int KIND>
void line_search_k(spirec_plan p, const float2* f, const float2* d, int step)
{
    k_line_search<KIND><<<vec_blocks(p->N), kVecThreads, 0, p->stream>>>(f, d, p->N, p->reg, step, slot(p, P_LS),
                                                                         p->counters + C_LS, p->scal);
}

template <int KIND>
void update_k(spirec_plan p, const float2* f_in, float2* f_out, const float2* d, float2* res, const float2* Td,
              float2* g, int first, double* Jout)
{
    if (first)
        k_update<true, KIND><<<vec_blocks(p->N), kVecThreads, 0, p->stream>>>(
            f_in, f_out, d, res, Td, p->D, g, p->N, p->reg, slot(p, P_UPD), p->counters + C_UPD, p->scal, Jout);
    else
        k_update<false, KIND><<<vec_blocks(p->N), kVecThreads, 0, p->stream>>>(
            f_in, f_out, d, res, Td, p->D, g, p->N, p->reg, slot(p, P_UPD), p->counters + C_UPD, p->scal, Jout);
}
}  // namespace

// phi fixed at compile time in the per-pixel work: one kernel per phi
int launch_line_search(spirec_plan p, const float2* f, const float2* d, int step)
{
    switch (p->reg.kind) {
    case SPIREC_PHI_HUBER: line_search_k<SPIREC_PHI_HUBER>(p, f, d, step); break;
    case SPIREC_PHI_HYPERBOLIC: line_search_k<SPIREC_PHI_HYPERBOLIC>(p, f, d, step); break;
    default: line_search_k<SPIREC_PHI_QUADRATIC>(p, f, d, step); break;
    }
    SPIREC_CK(cudaGetLastError());
    p->launches += 1;
    return SPIREC_OK;
}

int launch_update(spirec_plan p, const float2* f_in, float2* f_out, const float2* d, float2* res,
                  const float2* Td, float2* g, int first, double* Jout)
{
    switch (p->reg.kind) {
    case SPIREC_PHI_HUBER: update_k<SPIREC_PHI_HUBER>(p, f_in, f_out, d, res, Td, g, first, Jout); break;
    case SPIREC_PHI_HYPERBOLIC: update_k<SPIREC_PHI_HYPERBOLIC>(p, f_in, f_out, d, res, Td, g, first, Jout); break;
    default: update_k<SPIREC_PHI_QUADRATIC>(p, f_in, f_out, d, res, Td, g, first, Jout); break;
    }
    SPIREC_CK(cudaGetLastError());
    p->launches += 1;
    return SPIREC_OK;
}

// q2 = Re<d, T d> and the first line-search step
//   t1 = -(q1 + num0) / (2 q2 + den0)   (0 when the curvature is not > 0),
// as the fused row pass 3 of the FFT path computes them.
__global__ void k_q2_t1(const float2* d, const float2* Td, int64_t n, float2* parts, unsigned* counter,
                        double* scal)
{
    float v[1] = {0.f};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = __ldcg(d + i), b = __ldcg(Td + i);
        v[0] += fmaf(a.x, b.x, a.y * b.y);
    }
    FF bt[1];
    block_partial<1>(v, bt);
    store_parts<1>(bt, parts, kMaxParts);
    if (last_block(counter)) {
        FF t[1];
        sum_parts_ff<1>(parts, kMaxParts, gridDim.x, t);
        if (threadIdx.x == 0) {
            const double q2 = ff_to_double(t[0]);
            scal[S_Q2] = q2;
            const double curv = 2.0 * q2 + scal[S_DEN0];
            scal[S_T1] = curv > 0.0 ? -(scal[S_Q1] + scal[S_NUM0]) / curv : 0.0;
            *counter = 0u;
        }
    }
}

int launch_normal_direct(spirec_plan p, const float2* x, float2* Tx, bool dot_q2_t1)
{
    if (!p->ydir) {
        set_error("direct mode needs spirec_set_mode first");
        return SPIREC_ESTATE;
    }
    int rc;
    if ((rc = launch_forward(p, x, p->ydir)) != SPIREC_OK) return rc;
    if ((rc = launch_adjoint(p, p->ydir, Tx)) != SPIREC_OK) return rc;
    if (dot_q2_t1) {
        k_q2_t1<<<vec_blocks(p->N), kVecThreads, 0, p->stream>>>(x, Tx, (int64_t)p->N * p->N, slot(p, P_ROWC),
                                                                  p->counters + C_ROWC, p->scal);
        SPIREC_CK(cudaGetLastError());
        p->launches += 1;
    }
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
    a.res = p->res;
    a.D = p->D;
    a.reg = p->reg;
    a.parts = slot(p, P_ROWA);
    a.counter = p->counters + C_ROWA;
    a.scal = p->scal;
    // the new direction d, q1 and the t = 0 line-search sums (with the row
    // FFTs of d, which only the FFT path uses)
    if ((rc = launch_rows_fwd(p, nullptr, N, N, N, 1, &a)) != SPIREC_OK) return rc;
    if (p->mode == SPIREC_MODE_DIRECT) {
        if ((rc = launch_normal_direct(p, dk, p->Td, true)) != SPIREC_OK) return rc;
    } else {
        if ((rc = launch_cols(p, N, N)) != SPIREC_OK) return rc;
        CgPass c = a;
        c.parts = slot(p, P_ROWC);
        c.counter = p->counters + C_ROWC;
        if ((rc = launch_rows_inv(p, p->Td, 1, dk, &c, 0)) != SPIREC_OK) return rc;
    }
    for (int j = 1; j <= 2; ++j)
        if ((rc = launch_line_search(p, fin, dk, j)) != SPIREC_OK) return rc;
    return launch_update(p, fin, fout, dk, p->res, p->Td, p->g, 0, Jdev ? Jdev + k + 1 : nullptr);
}

}  // namespace spirec
