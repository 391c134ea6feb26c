// fft.cu -- shared-memory FFTs for the Toeplitz (Gram) operator, its kernel
// spectrum, and the row passes of the CG iteration that fuse into them.
//
// T x = H^H H x is a 2-D linear convolution of x with conj(G) (Appendix B).
// Embedded in an M x M circulant (M >= 2N-1; the "circular convolution" of
// section 3.4 holds only after this zero padding) it becomes
//     T x = crop_N( IFFT2( Chat .* FFT2( pad_M(x) ) ) ),
// with Chat = FFT2(c) / M^2 real because c[-y][-x] = conj c[y][x] (the point
// symmetry of G).  The apply runs in three passes over an N x M buffer X:
//   rows:    N row FFTs of the zero-padded rows (N inputs, M outputs),
//   columns: per column FFT (N nonzero inputs) -> * Chat -> IFFT, rows < N,
//   rows:    N row IFFTs, columns < N kept.
// Inside the CG iteration the first row pass also forms the new direction
// d = -g + beta d_old and the first line-search sums, and the last row pass
// forms q2 = Re<d, T d> and the first line-search step.  The bodies of the
// passes live in fft_device.cuh (shared with the persistent loop of
// cg_loop.cu); this file holds the stand-alone kernels and their launchers.
//
// FFTs are self-sorting Stockham transforms in shared memory.  For
// power-of-two M (the sizes the plan picks) the transform is compile-time:
// one radix-4 butterfly per thread per stage (plus one radix-2 stage for odd
// log2 M), values in registers between a read and a write phase.  Any other
// M = 2^a 3^b 5^c runs the runtime mixed-radix path with a ping-pong buffer.
// At M = 2048 and 4096, where every transform of the apply has at most M/2
// nonzero inputs and keeps at most M/2 outputs, the three passes instead
// split each transform into S = M / 1024 warp-sized 1024-point DFTs, one per
// output class k = r mod S (k_rows_fwd_split, k_cols_split,
// k_rows_inv_split).
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "fft_device.cuh"
#include "fft_reg.cuh"
#include "internal.cuh"
#include "phase.cuh"
#include "reduce.cuh"

namespace spirec {

bool make_fft_plan(int M, FftPlan* p)
{
    p->M = M;
    p->nstages = 0;
    int r = M;
    while (r > 1) {
        int rad;
        if (r % 4 == 0) rad = 4;
        else if (r % 2 == 0) rad = 2;
        else if (r % 3 == 0) rad = 3;
        else if (r % 5 == 0) rad = 5;
        else return false;
        if (p->nstages >= kMaxStages) return false;
        p->radix[p->nstages++] = rad;
        r /= rad;
    }
    return true;
}

namespace {

using namespace fftd;

// ------------------------------------------------------------- row pass 1

// MODE 0: row FFTs of `in` into X.  MODE 1 (CG): the rows of the new
// direction, with q1 and the first line-search sums reduced over the grid
// and finished by the last block into scal (see fft_device.cuh).
template <int MC, int MODE, int KIND = -1>
__global__ void __launch_bounds__(1024) k_rows_fwd(const float2* in, int ld_in, int n_in, int rows, float2* X, FftPlan fp,
                           const float2* __restrict__ tw, int rpc, CgPass c)
{
    extern __shared__ float2 sm[];
    float2* a = sm;
    float2* b = sm + rpc * seq_len<MC>(fp.M);
    const int r0 = blockIdx.x * rpc;
    const int nr = min(rpc, rows - r0);
    float beta = 0.f;
    bool restart = true;
    if (MODE == 1) {
        const double bd = c.scal[S_BETA];
        beta = (float)bd;
        restart = bd == 0.0;
    }
    float acc[3] = {0.f, 0.f, 0.f};
    rows_fwd_group<MC, MODE, KIND>(in, ld_in, n_in, r0, nr, rpc, X, fp, tw, c, beta, restart, a, b, acc);
    if (MODE == 1) {
        FF bt[3];
        block_partial<3>(acc, bt);
        store_parts<3>(bt, c.parts, kMaxParts);
        if (last_block(c.counter)) {
            FF t[3];
            sum_parts_ff<3>(c.parts, kMaxParts, gridDim.x, t);
            if (threadIdx.x == 0) {
                c.scal[S_Q1] = ff_to_double(t[0]);
                c.scal[S_NUM0] = ff_to_double(t[1]);
                c.scal[S_DEN0] = ff_to_double(t[2]);
                *c.counter = 0u;
            }
        }
    }
}

// ------------------------------------------------------------- row pass 3

// Row IFFTs of X, first n_out columns to out.  With dotx: s = Re<dotx, out>
// over the grid; MODE 0 stores it in scal[dot_scalar]; MODE 1 (CG) stores
// q2 = s and the first line-search step
//   t1 = -(q1 + num0) / (2 q2 + den0)   (0 when the curvature is not > 0).
template <int MC, int MODE>
__global__ void __launch_bounds__(1024) k_rows_inv(const float2* X, int rows, float2* out, int n_out, FftPlan fp,
                           const float2* __restrict__ tw, int rpc, const float2* dotx, CgPass c,
                           int dot_scalar)
{
    extern __shared__ float2 sm[];
    float2* a = sm;
    float2* b = sm + rpc * seq_len<MC>(fp.M);
    const int r0 = blockIdx.x * rpc;
    const int nr = min(rpc, rows - r0);
    float acc = 0.f;
    rows_inv_group<MC>(X, r0, nr, rpc, out, n_out, fp, tw, dotx, a, b, acc);
    if (dotx) {
        float v[1] = {acc};
        FF bt[1];
        block_partial<1>(v, bt);
        store_parts<1>(bt, c.parts, kMaxParts);
        if (last_block(c.counter)) {
            FF t[1];
            sum_parts_ff<1>(c.parts, kMaxParts, gridDim.x, t);
            if (threadIdx.x == 0) {
                const double s = ff_to_double(t[0]);
                if (MODE == 0) {
                    c.scal[dot_scalar] = s;
                } else {
                    c.scal[S_Q2] = s;
                    const double curv = 2.0 * s + c.scal[S_DEN0];
                    c.scal[S_T1] = curv > 0.0 ? -(c.scal[S_Q1] + c.scal[S_NUM0]) / curv : 0.0;
                }
                *c.counter = 0u;
            }
        }
    }
}

// ------------------------------------------------------------- column pass

template <int MC>
__global__ void __launch_bounds__(1024) k_cols_filter(float2* X, int n_in, int n_out, FftPlan fp, const float2* __restrict__ tw,
                              const float* __restrict__ Chat, int cpc)
{
    extern __shared__ float2 sm[];
    const int ld = seq_len<MC>(fp.M) + 4;
    const int x0 = blockIdx.x * cpc;
    cols_group<MC>(X, n_in, n_out, x0, min(cpc, fp.M - x0), cpc, fp, tw, Chat, sm, sm + cpc * ld);
}

// ----------------------------------------- column pass, M = 1024 S >= 2048

// One warp, the 1024-point DFT (conjugate twiddles when INV) of the sequence
// whose element lane + 32 j is in x[j], as four steps: DFT over the
// registers, twiddles w1024^(lane k1) from t2, transpose through this warp's
// area (32 x 33), DFT over the registers.  Element lane + 32 k2 of the result
// ends in x[bitrev5(k2)].  t2[k1 * 32 + l] = w1024^(k1 l).
template <bool INV>
__device__ __forceinline__ void dft1024_warp(float2 (&x)[32], float2* area, const float2* t2, int lane)
{
    freg::dft32_dif<INV>(x);
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) {
        const float2 w = t2[k1 * 32 + lane];
        area[k1 * 33 + lane] = cmul(x[freg::bitrev5(k1)], INV ? conjf2(w) : w);
    }
    __syncwarp();
#pragma unroll
    for (int l = 0; l < 32; ++l) x[l] = area[lane * 33 + l];
    __syncwarp();
    freg::dft32_dif<INV>(x);
}

// x[k] <-> x[bitrev5(k)]: the bit-reversed register order to the natural one
// (compile-time indices: a renaming, no data moves).
__device__ __forceinline__ void unreverse32(float2 (&x)[32])
{
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const int b = freg::bitrev5(k);
        if (k < b) {
            const float2 t = x[k];
            x[k] = x[b];
            x[b] = t;
        }
    }
}

// The split passes run 8 warps a CTA and two CTAs an SM, so that one CTA's
// loads overlap the other's transforms.
constexpr int kSplitWarps = 8;
constexpr int kSplitThreads = 32 * kSplitWarps;
constexpr int kSplitCtasPerSm = 16 / kSplitWarps;
// The inverse row pass has no staging buffer (76 KB of shared memory a CTA),
// so three CTAs fit an SM; its DFTs fit 85 registers a thread without spills.
constexpr int kSplitInvCtasPerSm = 3;
// Warp area of the column pass: 32 x 33 for the four-step DFT plus 2, so that
// the S areas of one column start 8 (S = 4) or 4 (S = 2) float2 banks after
// those of the previous column, and the combine step, whose neighbouring
// threads read neighbouring columns, hits distinct banks.
constexpr int kSplitArea = 1058;

// Input m (m < 1024) of the 1024-point DFT that gives the outputs k = r mod S
// of an M = 1024 S point DFT of x (x zero from M/2 on):
//   z_r[m] = w_M^(r m) sum_{t < S/2} x[m + 1024 t] w_S^(r t),
// as w_M^(r (m + 1024 t)) = w_M^(r m) w_S^(r t).  For S = 4 the factor
// w_4^r = (-i)^r is applied exactly (a swap and sign changes).
template <int S>
__device__ __forceinline__ float2 fold_input(const float2* x, int m, int r, const float2* __restrict__ tw)
{
    float2 z = x[m];
    if constexpr (S == 4) {
        const float2 v = x[m + 1024];
        const float2 rv = r == 0 ? v : r == 1 ? make_float2(v.y, -v.x) : r == 2 ? make_float2(-v.x, -v.y)
                                                                                : make_float2(-v.y, v.x);
        z = freg::add(z, rv);
    }
    return r == 0 ? z : cmul(z, __ldg(tw + r * m));
}

// Output n (n < M/2) of the inverse M-point DFT from the S inverse 1024-point
// DFTs u_r of the classes k = r mod S (u_r at u + r * stride, index n mod
// 1024 applied by the caller): sum_r w_M^(-r n) u_r, by Horner's rule in
// conj(w_M^n).
template <int S>
__device__ __forceinline__ float2 combine_output(const float2* u, int stride, int n, const float2* __restrict__ tw)
{
    const float2 c = conjf2(__ldg(tw + n));
    float2 y = u[(S - 1) * stride];
#pragma unroll
    for (int r = S - 2; r >= 0; --r) y = freg::add(u[r * stride], cmul(c, y));
    return y;
}

// Stride of a staged column of k_cols_split<S>: the 8 / S columns of one
// row piece land on distinct banks (offsets 8 float2 apart for two columns,
// 4 for four).
template <int S>
__host__ __device__ constexpr int cols_split_ld() { return 512 * S + (S == 4 ? 8 : 4); }

// Shared memory of k_cols_split<S>: the warps' areas, whose start the staged
// columns share (they are dead once every warp has folded its column into
// registers), then the 32 x 32 twiddles: 76 KB, three CTAs an SM.
template <int S>
constexpr size_t cols_split_smem()
{
    const size_t stage = (size_t)(kSplitWarps / S) * cols_split_ld<S>(), areas = (size_t)kSplitWarps * kSplitArea;
    return ((stage > areas ? stage : areas) + 1024) * sizeof(float2);
}
constexpr int kSplitColCtasPerSm = 3;

// The Toeplitz column pass for M = 1024 S (S = 2, 4) when at most M/2 rows
// are nonzero and at most M/2 are kept (n_in, n_out <= M/2, always the case
// for N x N images): column FFT * Chat * IFFT with every 1024-point DFT in
// one warp's registers.  X[S k + r] = DFT1024(z_r)[k] with
// z_r[m] = sum_t x[m + 1024 t] w_M^(r (m + 1024 t)) (t < S/2, the input
// folded to 1024 points), so warp r of a column computes the outputs
// k = r mod S; after the spectrum and the inverse 1024-point DFT u_r, the
// column's rows are y[n] = sum_r w_M^(-r n) u_r[n mod 1024], summed in a fixed
// order.  8 / S columns a group, staged from X as row pieces of 8 / S
// neighbouring columns; CTAs loop over the groups.  tw[e] = w_M^e.
template <int S>
__global__ void __launch_bounds__(kSplitThreads, kSplitColCtasPerSm)
k_cols_split(float2* X, int n_in, int n_out, const float2* __restrict__ tw, const float* __restrict__ Chat)
{
    constexpr int M = 1024 * S, C = kSplitWarps / S, H = M / 2, LDS = cols_split_ld<S>();
    static_assert(C * LDS <= kSplitWarps * kSplitArea, "the staged columns fit in the areas");
    extern __shared__ float2 sm[];
    float2* areas = sm;
    float2* stage = sm;  // shares the areas' start
    float2* t2 = areas + kSplitWarps * kSplitArea;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cc = warp / S, r = warp - cc * S;
    for (int e = tid; e < 1024; e += kSplitThreads) t2[e] = __ldg(tw + ((S * (e >> 5) * (e & 31)) & (M - 1)));
    for (int x0 = blockIdx.x * C; x0 < M; x0 += gridDim.x * C) {
#pragma unroll 8
        for (int e = tid; e < C * H; e += kSplitThreads) {
            const int y = e / C, c = e - y * C;
            stage[c * LDS + y] = y < n_in ? __ldcg(X + (int64_t)y * M + x0 + c) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        // the warp's folded, twiddled input into registers; then every warp
        // has read the stage, and the areas may overwrite it
        float2 x[32];
        {
            const float2* col = stage + cc * LDS;
#pragma unroll
            for (int j = 0; j < 32; ++j) x[j] = fold_input<S>(col, lane + 32 * j, r, tw);
        }
        __syncthreads();
        float2* area = areas + warp * kSplitArea;
        dft1024_warp<false>(x, area, t2, lane);  // X[S (lane + 32 k2) + r] in x[bitrev5(k2)]
        unreverse32(x);
        {
            const float* ch = Chat + (int64_t)(x0 + cc) * M + r + S * lane;
#pragma unroll
            for (int k2 = 0; k2 < 32; ++k2) {
                const float h = __ldg(ch + 32 * S * k2);
                x[k2] = make_float2(x[k2].x * h, x[k2].y * h);
            }
        }
        dft1024_warp<true>(x, area, t2, lane);  // u_r[lane + 32 m2] in x[bitrev5(m2)]
#pragma unroll
        for (int m2 = 0; m2 < 32; ++m2) area[lane + 32 * m2] = x[freg::bitrev5(m2)];
        __syncthreads();
#pragma unroll 4
        for (int e = tid; e < C * n_out; e += kSplitThreads) {
            const int y = e / C, c = e - y * C;
            X[(int64_t)y * M + x0 + c] = combine_output<S>(areas + c * S * kSplitArea + (y & 1023), kSplitArea, y, tw);
        }
        __syncthreads();  // the next group refills the stage and the areas
    }
}

// ------------------------------------------- row passes, M = 1024 S >= 2048

// Warp areas of the split row passes: 32 x 33 for the four-step DFT, padded
// so that whole-row copies, whose neighbouring elements k = S j + r live in
// the S areas of a row at j, hit distinct banks (area stride = 4 or 8 mod 16).
template <int S>
__host__ __device__ constexpr int row_area() { return 1056 + (S == 4 ? 4 : 8); }

// Shared memory of the split row passes: (pass 1 only) the staged rows, then
// the warps' areas and the 32 x 32 twiddles.
template <int S, bool STAGE>
constexpr size_t rows_split_smem()
{
    return ((STAGE ? (size_t)(kSplitWarps / S) * (512 * S + 4) : 0) + kSplitWarps * row_area<S>() + 1024) * sizeof(float2);
}

// Row pass 1 for M = 1024 S (S = 2, 4) with at most M/2 nonzero inputs
// (n_in <= M/2): the rows (MODE 1: the new direction d = -g + beta d_old,
// written to d_new, with q1 and the first line-search sums as in
// rows_fwd_group) staged in shared memory, then warp r of a row computes the
// outputs k = r mod S of its 1024-point DFT from the folded input
// sum_t x[m + 1024 t] w_M^(r (m + 1024 t)), and the block writes whole rows
// of X.  8 / S rows a group; CTAs loop over the groups.
template <int S, int MODE, int KIND>
__global__ void __launch_bounds__(kSplitThreads, kSplitCtasPerSm)
k_rows_fwd_split(const float2* in, int ld_in, int n_in, int rows, float2* X, const float2* __restrict__ tw,
                 CgPass c)
{
    constexpr int M = 1024 * S, R = kSplitWarps / S, H = M / 2, LDS = H + 4, A = row_area<S>();
    extern __shared__ float2 sm[];
    float2* stage = sm;
    float2* areas = stage + R * LDS;
    float2* t2 = areas + kSplitWarps * A;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp / S, r = warp - q * S;
    for (int e = tid; e < 1024; e += kSplitThreads) t2[e] = __ldg(tw + ((S * (e >> 5) * (e & 31)) & (M - 1)));
    float beta = 0.f;
    bool restart = true;
    if (MODE == 1) {
        const double bd = c.scal[S_BETA];
        beta = (float)bd;
        restart = bd == 0.0;
    }
    const int N = n_in;
    float acc[3] = {0.f, 0.f, 0.f};
    for (int r0 = blockIdx.x * R; r0 < rows; r0 += gridDim.x * R) {
        const int nr = min(R, rows - r0);
#pragma unroll 4
        for (int e = tid; e < R * H; e += kSplitThreads) {
            const int qq = e / H, m = e - qq * H;
            float2 v = make_float2(0.f, 0.f);
            if (qq < nr && m < N) {
                const int64_t o = (int64_t)(r0 + qq) * ld_in + m;
                if (MODE == 0) {
                    v = __ldcg(in + o);
                } else {
                    v = new_direction(__ldcg(c.g + o), __ldcg(c.d_old + o), beta, restart);
                    c.d_new[o] = v;
                }
            }
            stage[qq * LDS + m] = v;
        }
        __syncthreads();
        if (MODE == 1) {
            const Reg reg = c.reg;
#pragma unroll 4
            for (int e = tid; e < nr * N; e += kSplitThreads) {
                const int qq = e / N, m = e - qq * N;
                const int n = r0 + qq;
                const int64_t o = (int64_t)n * N + m;
                const bool has_r = m + 1 < N, has_d = n + 1 < N;
                const int64_t od = has_d ? o + N : o;
                const float2 dn = stage[qq * LDS + m];
                const float2 dr = stage[qq * LDS + (has_r ? m + 1 : m)];
                const float2 fp_ = __ldcg(c.f + o), fr = __ldcg(c.f + (has_r ? o + 1 : o)), fd = __ldcg(c.f + od);
                const float2 gd = __ldcg(c.g + od), dold_d = __ldcg(c.d_old + od);
                acc[0] += 2.f * redot(dn, __ldcg(c.res + o));
                if (reg.lambda1 != 0.f) {
                    {
                        const float2 w = f2sub(dr, dn);
                        const float2 z = f2sub(fr, fp_);
                        const float bw =
                            has_r ? reg.lambda1 * phi_weight_k<KIND>(reg.kind, reg.alpha1, redot(z, z)) : 0.f;
                        acc[1] = fmaf(bw, redot(z, w), acc[1]);
                        acc[2] = fmaf(bw, redot(w, w), acc[2]);
                    }
                    {
                        const float2 dd = new_direction(gd, dold_d, beta, restart);
                        const float2 w = f2sub(dd, dn);
                        const float2 z = f2sub(fd, fp_);
                        const float bw =
                            has_d ? reg.lambda1 * phi_weight_k<KIND>(reg.kind, reg.alpha1, redot(z, z)) : 0.f;
                        acc[1] = fmaf(bw, redot(z, w), acc[1]);
                        acc[2] = fmaf(bw, redot(w, w), acc[2]);
                    }
                }
                if (reg.lambda0 != 0.f) {
                    const float bw = reg.lambda0 * phi_weight_k<KIND>(reg.kind, reg.alpha0, redot(fp_, fp_));
                    acc[1] = fmaf(bw, redot(fp_, dn), acc[1]);
                    acc[2] = fmaf(bw, redot(dn, dn), acc[2]);
                }
            }
        }
        if (q < nr) {
            float2* area = areas + warp * A;
            const float2* row = stage + q * LDS;
#pragma unroll 4
            for (int m = lane; m < 1024; m += 32) area[m] = fold_input<S>(row, m, r, tw);
            __syncwarp();
            float2 x[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) x[j] = area[lane + 32 * j];
            __syncwarp();
            dft1024_warp<false>(x, area, t2, lane);
#pragma unroll
            for (int k2 = 0; k2 < 32; ++k2) area[lane + 32 * k2] = x[freg::bitrev5(k2)];
        }
        __syncthreads();
        for (int e = tid; e < nr * M; e += kSplitThreads) {
            const int qq = e / M, kk = e - qq * M;
            X[(int64_t)(r0 + qq) * M + kk] = areas[(qq * S + (kk & (S - 1))) * A + kk / S];
        }
        __syncthreads();  // the next group refills the stage and the areas
    }
    if (MODE == 1) {
        FF bt[3];
        block_partial<3>(acc, bt);
        store_parts<3>(bt, c.parts, kMaxParts);
        if (last_block(c.counter)) {
            FF t[3];
            sum_parts_ff<3>(c.parts, kMaxParts, gridDim.x, t);
            if (threadIdx.x == 0) {
                c.scal[S_Q1] = ff_to_double(t[0]);
                c.scal[S_NUM0] = ff_to_double(t[1]);
                c.scal[S_DEN0] = ff_to_double(t[2]);
                *c.counter = 0u;
            }
        }
    }
}

// Row pass 3 for M = 1024 S (S = 2, 4), n_out <= M/2: each row of X copied
// whole into the S warp areas (element S j + r to area r at j), warp r's
// inverse 1024-point DFT u_r, and out[m] = sum_r w_M^(-r m) u_r[m mod 1024]
// in a fixed order; with dotx the same grid sum and scalars as k_rows_inv.
template <int S, int MODE>
__global__ void __launch_bounds__(kSplitThreads, kSplitInvCtasPerSm)
k_rows_inv_split(const float2* X, int rows, float2* out, int n_out, const float2* __restrict__ tw,
                 const float2* dotx, CgPass c, int dot_scalar)
{
    constexpr int M = 1024 * S, R = kSplitWarps / S, A = row_area<S>();
    extern __shared__ float2 sm[];
    float2* areas = sm;
    float2* t2 = areas + kSplitWarps * A;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp / S;
    for (int e = tid; e < 1024; e += kSplitThreads) t2[e] = __ldg(tw + ((S * (e >> 5) * (e & 31)) & (M - 1)));
    float acc = 0.f;
    for (int r0 = blockIdx.x * R; r0 < rows; r0 += gridDim.x * R) {
        const int nr = min(R, rows - r0);
#pragma unroll 8
        for (int e = tid; e < nr * M; e += kSplitThreads) {
            const int qq = e / M, kk = e - qq * M;
            areas[(qq * S + (kk & (S - 1))) * A + kk / S] = __ldcg(X + (int64_t)(r0 + qq) * M + kk);
        }
        __syncthreads();
        if (q < nr) {
            float2* area = areas + warp * A;
            float2 x[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) x[j] = area[lane + 32 * j];
            __syncwarp();
            dft1024_warp<true>(x, area, t2, lane);  // u_r[lane + 32 m2] in x[bitrev5(m2)]
#pragma unroll
            for (int m2 = 0; m2 < 32; ++m2) area[lane + 32 * m2] = x[freg::bitrev5(m2)];
        }
        __syncthreads();
#pragma unroll 4
        for (int e = tid; e < nr * n_out; e += kSplitThreads) {
            const int qq = e / n_out, m = e - qq * n_out;
            const float2 y = combine_output<S>(areas + qq * S * A + (m & 1023), A, m, tw);
            const int64_t o = (int64_t)(r0 + qq) * n_out + m;
            out[o] = y;
            if (dotx) acc += redot(__ldcg(dotx + o), y);
        }
        __syncthreads();
    }
    if (dotx) {
        float v[1] = {acc};
        FF bt[1];
        block_partial<1>(v, bt);
        store_parts<1>(bt, c.parts, kMaxParts);
        if (last_block(c.counter)) {
            FF t[1];
            sum_parts_ff<1>(c.parts, kMaxParts, gridDim.x, t);
            if (threadIdx.x == 0) {
                const double sv = ff_to_double(t[0]);
                if (MODE == 0) {
                    c.scal[dot_scalar] = sv;
                } else {
                    c.scal[S_Q2] = sv;
                    const double curv = 2.0 * sv + c.scal[S_DEN0];
                    c.scal[S_T1] = curv > 0.0 ? -(c.scal[S_Q1] + c.scal[S_NUM0]) / curv : 0.0;
                }
                *c.counter = 0u;
            }
        }
    }
}

// Column FFTs of the M x M circulant and the real spectrum:
// Chat[x][ky] = Re(FFT2 c)[ky][x] / M^2.
template <int MC>
__global__ void __launch_bounds__(1024) k_cols_spectrum(const float2* cwork, FftPlan fp, const float2* __restrict__ tw,
                                float* Chat, int cpc)
{
    extern __shared__ float2 sm[];
    const int M = fp.M;
    const int ld = seq_len<MC>(M) + 4;
    float2* a = sm;
    float2* b = sm + cpc * ld;
    const int x0 = blockIdx.x * cpc;
    const int nc = min(cpc, M - x0);
    for (int e = threadIdx.x; e < cpc * M; e += blockDim.x) {
        const int y = e / cpc, cc = e - y * cpc;
        a[cc * ld + sidx<MC>(y)] = cc < nc ? cwork[(int64_t)y * M + x0 + cc] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* res = fft_block<MC, false>(a, b, fp, cpc, ld, tw);
    const float inv = 1.0f / ((float)M * (float)M);
    for (int e = threadIdx.x; e < nc * M; e += blockDim.x) {
        const int cc = e / M, ky = e - cc * M;
        Chat[(int64_t)(x0 + cc) * M + ky] = res[cc * ld + sidx<MC>(ky)].x * inv;
    }
}

// c[y][x] = K[v][u] = conj G_{u,v} with v = y (y < N) or y - M (y > M - N),
// u likewise from x; zero where |u| or |v| >= N.  G holds u >= 0; the rest is
// G_{u,v} = conj G_{-u,-v}.
__global__ void __launch_bounds__(256) k_embed(const float2* __restrict__ G, int N, int M, float2* cwork)
{
    // one 32 x 32 tile of cwork through shared memory: G is read along its
    // rows (the lags v of one u) and cwork written along its rows (x)
    __shared__ float2 tile[32][33];  // [x - x0][y - y0]
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const int W = 2 * N - 1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int x = x0 + ty + 8 * k, y = y0 + tx;
        float2 c = make_float2(0.f, 0.f);
        if (x < M && y < M) {
            const int v = y < N ? y : (y > M - N ? y - M : INT32_MIN);
            const int u = x < N ? x : (x > M - N ? x - M : INT32_MIN);
            if (v != INT32_MIN && u != INT32_MIN) {
                if (u >= 0) {
                    const float2 g = G[(int64_t)u * W + (v + N - 1)];
                    c = make_float2(g.x, -g.y);
                } else {
                    c = G[(int64_t)(-u) * W + (-v + N - 1)];
                }
            }
        }
        tile[ty + 8 * k][tx] = c;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int x = x0 + tx, y = y0 + ty + 8 * k;
        if (x < M && y < M) cwork[(int64_t)y * M + x] = tile[tx][ty + 8 * k];
    }
}

// ------------------------------------------------------------- launch shapes

constexpr int kFftSmemCap = 200 * 1024;

struct Shape {
    int per_cta;  // rows or columns per CTA
    int threads;
    size_t smem;
};

// Compile-time path: nseq * M / 4 threads (<= 1024), single buffer.
// Runtime path: 256 threads, ping-pong buffers.
Shape row_shape(int M, bool pow2)
{
    if (pow2) {
        const int nb = M / 4;
        const int rpc = nb >= 256 ? 1 : 256 / nb;
        return Shape{rpc, rpc * nb, (size_t)rpc * seq_len<1>(M) * sizeof(float2)};
    }
    const int rpc = M >= 1024 ? 1 : 1024 / M;
    return Shape{rpc, 256, 2 * (size_t)rpc * M * sizeof(float2)};
}

Shape col_shape(int M, bool pow2)
{
    if (pow2) {
        const int nb = M / 4;
        int cpc = nb >= 1024 ? 1 : 1024 / nb;
        const size_t ld = seq_len<1>(M) + 4;
        while (cpc > 1 && (size_t)cpc * ld * sizeof(float2) > (size_t)kFftSmemCap) cpc /= 2;
        return Shape{cpc, cpc * nb, (size_t)cpc * ld * sizeof(float2)};
    }
    int cpc = M >= 1024 ? 4 : (M >= 512 ? 8 : 16);
    while (cpc > 1 && 2 * (size_t)cpc * (M + 4) * sizeof(float2) > (size_t)kFftSmemCap) --cpc;
    return Shape{cpc, 256, 2 * (size_t)cpc * (M + 4) * sizeof(float2)};
}

template <int MC>
int set_attrs()
{
    const int bytes = kFftSmemCap;
    SPIREC_CK(cudaFuncSetAttribute(k_rows_fwd<MC, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SPIREC_CK(cudaFuncSetAttribute(k_rows_fwd<MC, 1, SPIREC_PHI_HUBER>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SPIREC_CK(cudaFuncSetAttribute(k_rows_fwd<MC, 1, SPIREC_PHI_HYPERBOLIC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   bytes));
    SPIREC_CK(cudaFuncSetAttribute(k_rows_fwd<MC, 1, SPIREC_PHI_QUADRATIC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   bytes));
    SPIREC_CK(cudaFuncSetAttribute(k_rows_inv<MC, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SPIREC_CK(cudaFuncSetAttribute(k_rows_inv<MC, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SPIREC_CK(cudaFuncSetAttribute(k_cols_filter<MC>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SPIREC_CK(cudaFuncSetAttribute(k_cols_spectrum<MC>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    return SPIREC_OK;
}

template <int S>
int set_split_row_attrs()
{
    const int fb = (int)rows_split_smem<S, true>(), ib = (int)rows_split_smem<S, false>();
    SPIREC_CK(cudaFuncSetAttribute(k_rows_fwd_split<S, 0, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, fb));
    SPIREC_CK(cudaFuncSetAttribute(k_rows_fwd_split<S, 1, SPIREC_PHI_HUBER>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, fb));
    SPIREC_CK(cudaFuncSetAttribute(k_rows_fwd_split<S, 1, SPIREC_PHI_HYPERBOLIC>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, fb));
    SPIREC_CK(cudaFuncSetAttribute(k_rows_fwd_split<S, 1, SPIREC_PHI_QUADRATIC>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, fb));
    SPIREC_CK(cudaFuncSetAttribute(k_rows_inv_split<S, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, ib));
    SPIREC_CK(cudaFuncSetAttribute(k_rows_inv_split<S, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, ib));
    return SPIREC_OK;
}

// Calls f.template operator()<MC>() with the compile-time size for M, or
// MC = 0 for sizes without a specialisation.
template <typename F>
int with_size(int M, F&& f)
{
    switch (M) {
    case 16: return f.template operator()<16>();
    case 32: return f.template operator()<32>();
    case 64: return f.template operator()<64>();
    case 128: return f.template operator()<128>();
    case 256: return f.template operator()<256>();
    case 512: return f.template operator()<512>();
    case 1024: return f.template operator()<1024>();
    case 2048: return f.template operator()<2048>();
    case 4096: return f.template operator()<4096>();
    default: return f.template operator()<0>();
    }
}

bool is_pow2_specialised(int M) { return M >= 16 && M <= 4096 && (M & (M - 1)) == 0; }

CgPass plain_pass(spirec_plan p, int slot, unsigned* counter)
{
    CgPass c{};
    c.parts = reinterpret_cast<float2*>(p->part) + (size_t)slot * kMaxParts;
    c.counter = counter;
    c.scal = p->scal;
    c.reg = p->reg;
    return c;
}

struct AttrAll {
    template <int MC>
    int operator()() { return MC > 0 ? set_attrs<MC>() : SPIREC_OK; }
};

struct LaunchRowsFwd {
    spirec_plan p;
    const float2* in;
    int ld_in, n_in, rows, mode, blocks;
    Shape s;
    CgPass c;
    int split_grid;  // CTAs of the split passes (M = 2048, 4096): two an SM
    template <int S, int MODE, int KIND>
    void split(int grid)
    {
        k_rows_fwd_split<S, MODE, KIND><<<grid, kSplitThreads, rows_split_smem<S, true>(), p->stream>>>(
            in, ld_in, n_in, rows, p->X, p->twiddle, c);
    }
    template <int MC>
    int operator()()
    {
        if constexpr (MC == 2048 || MC == 4096) {
            constexpr int S = MC / 1024;
            if (2 * n_in <= MC) {
                const int groups = (rows + kSplitWarps / S - 1) / (kSplitWarps / S);
                const int grid = groups < split_grid ? groups : split_grid;
                if (mode == 0) split<S, 0, -1>(grid);
                else if (c.reg.kind == SPIREC_PHI_HUBER) split<S, 1, SPIREC_PHI_HUBER>(grid);
                else if (c.reg.kind == SPIREC_PHI_HYPERBOLIC) split<S, 1, SPIREC_PHI_HYPERBOLIC>(grid);
                else split<S, 1, SPIREC_PHI_QUADRATIC>(grid);
                SPIREC_CK(cudaGetLastError());
                p->launches += 1;
                return SPIREC_OK;
            }
        }
        if (mode == 0)
            k_rows_fwd<MC, 0><<<blocks, s.threads, s.smem, p->stream>>>(in, ld_in, n_in, rows, p->X, p->fft,
                                                                        p->twiddle, s.per_cta, c);
        else if (c.reg.kind == SPIREC_PHI_HUBER)  // phi fixed at compile time in the line-search sums
            k_rows_fwd<MC, 1, SPIREC_PHI_HUBER><<<blocks, s.threads, s.smem, p->stream>>>(
                in, ld_in, n_in, rows, p->X, p->fft, p->twiddle, s.per_cta, c);
        else if (c.reg.kind == SPIREC_PHI_HYPERBOLIC)
            k_rows_fwd<MC, 1, SPIREC_PHI_HYPERBOLIC><<<blocks, s.threads, s.smem, p->stream>>>(
                in, ld_in, n_in, rows, p->X, p->fft, p->twiddle, s.per_cta, c);
        else
            k_rows_fwd<MC, 1, SPIREC_PHI_QUADRATIC><<<blocks, s.threads, s.smem, p->stream>>>(
                in, ld_in, n_in, rows, p->X, p->fft, p->twiddle, s.per_cta, c);
        SPIREC_CK(cudaGetLastError());
        p->launches += 1;
        return SPIREC_OK;
    }
};

struct LaunchCols {
    spirec_plan p;
    int n_in, n_out, blocks;
    Shape s;
    template <int MC>
    int operator()()
    {
        if constexpr (MC == 2048 || MC == 4096) {
            constexpr int S = MC / 1024;
            if (2 * n_in <= MC && 2 * n_out <= MC) {
                int sms = 0;
                if (device_sms(&sms) != SPIREC_OK) return SPIREC_ECUDA;
                const int groups = MC / (kSplitWarps / S);
                const int cap = kSplitColCtasPerSm * sms;
                k_cols_split<S><<<groups < cap ? groups : cap, kSplitThreads, cols_split_smem<S>(), p->stream>>>(
                    p->X, n_in, n_out, p->twiddle, p->Chat);
                SPIREC_CK(cudaGetLastError());
                p->launches += 1;
                return SPIREC_OK;
            }
        }
        k_cols_filter<MC><<<blocks, s.threads, s.smem, p->stream>>>(p->X, n_in, n_out, p->fft, p->twiddle,
                                                                    p->Chat, s.per_cta);
        SPIREC_CK(cudaGetLastError());
        p->launches += 1;
        return SPIREC_OK;
    }
};

struct LaunchRowsInv {
    spirec_plan p;
    float2* out;
    int mode;
    const float2* dotx;
    int dot_scalar, blocks;
    Shape s;
    CgPass c;
    int split_grid;
    template <int MC>
    int operator()()
    {
        if constexpr (MC == 2048 || MC == 4096) {
            constexpr int S = MC / 1024;
            if (2 * p->N <= MC) {
                const int groups = (p->N + kSplitWarps / S - 1) / (kSplitWarps / S);
                const int grid = groups < split_grid ? groups : split_grid;
                if (mode == 0)
                    k_rows_inv_split<S, 0><<<grid, kSplitThreads, rows_split_smem<S, false>(), p->stream>>>(
                        p->X, p->N, out, p->N, p->twiddle, dotx, c, dot_scalar);
                else
                    k_rows_inv_split<S, 1><<<grid, kSplitThreads, rows_split_smem<S, false>(), p->stream>>>(
                        p->X, p->N, out, p->N, p->twiddle, dotx, c, dot_scalar);
                SPIREC_CK(cudaGetLastError());
                p->launches += 1;
                return SPIREC_OK;
            }
        }
        if (mode == 0)
            k_rows_inv<MC, 0><<<blocks, s.threads, s.smem, p->stream>>>(p->X, p->N, out, p->N, p->fft,
                                                                        p->twiddle, s.per_cta, dotx, c, dot_scalar);
        else
            k_rows_inv<MC, 1><<<blocks, s.threads, s.smem, p->stream>>>(p->X, p->N, out, p->N, p->fft,
                                                                        p->twiddle, s.per_cta, dotx, c, dot_scalar);
        SPIREC_CK(cudaGetLastError());
        p->launches += 1;
        return SPIREC_OK;
    }
};

struct LaunchSpectrum {
    spirec_plan p;
    Shape rs, cs;
    template <int MC>
    int operator()()
    {
        const int M = p->M;
        CgPass c{};
        // rows of the circulant, in place (each block reads its rows fully first)
        k_rows_fwd<MC, 0><<<(M + rs.per_cta - 1) / rs.per_cta, rs.threads, rs.smem, p->stream>>>(
            p->cwork, M, M, M, p->cwork, p->fft, p->twiddle, rs.per_cta, c);
        SPIREC_CK(cudaGetLastError());
        k_cols_spectrum<MC><<<(M + cs.per_cta - 1) / cs.per_cta, cs.threads, cs.smem, p->stream>>>(
            p->cwork, p->fft, p->twiddle, p->Chat, cs.per_cta);
        SPIREC_CK(cudaGetLastError());
        p->launches += 2;
        return SPIREC_OK;
    }
};

}  // namespace

int fft_setup_attributes(int)
{
    int rc;
    if ((rc = set_attrs<0>()) != SPIREC_OK) return rc;
    SPIREC_CK(cudaFuncSetAttribute(k_cols_split<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)cols_split_smem<2>()));
    SPIREC_CK(cudaFuncSetAttribute(k_cols_split<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)cols_split_smem<4>()));
    if ((rc = set_split_row_attrs<2>()) != SPIREC_OK) return rc;
    if ((rc = set_split_row_attrs<4>()) != SPIREC_OK) return rc;
    for (int M = 16; M <= 4096; M *= 2)
        if ((rc = with_size(M, AttrAll{})) != SPIREC_OK) return rc;
    return SPIREC_OK;
}

int launch_rows_fwd(spirec_plan p, const float2* in, int ld_in, int n_in, int rows, int mode,
                    const CgPass* cg)
{
    const int M = p->M;
    const Shape s = row_shape(M, is_pow2_specialised(M));
    const int blocks = (rows + s.per_cta - 1) / s.per_cta;
    if (mode == 1 && blocks > kMaxParts) {
        set_error("too many row blocks");
        return SPIREC_EUNSUPPORTED;
    }
    const CgPass c = cg ? *cg : plain_pass(p, 0, nullptr);
    int sms = 0;
    if (device_sms(&sms) != SPIREC_OK) return SPIREC_ECUDA;
    return with_size(M, LaunchRowsFwd{p, in, ld_in, n_in, rows, mode, blocks, s, c, kSplitCtasPerSm * sms});
}

int launch_cols(spirec_plan p, int n_in, int n_out)
{
    const int M = p->M;
    const Shape s = col_shape(M, is_pow2_specialised(M));
    const int blocks = (M + s.per_cta - 1) / s.per_cta;
    return with_size(M, LaunchCols{p, n_in, n_out, blocks, s});
}

int launch_rows_inv(spirec_plan p, float2* out, int mode, const float2* dotx, const CgPass* cg,
                    int dot_scalar)
{
    const int M = p->M, N = p->N;
    const Shape s = row_shape(M, is_pow2_specialised(M));
    const int blocks = (N + s.per_cta - 1) / s.per_cta;
    if (dotx && blocks > kMaxParts) {
        set_error("too many row blocks");
        return SPIREC_EUNSUPPORTED;
    }
    const CgPass c = cg ? *cg : plain_pass(p, P_MISC, p->counters + C_MISC);
    int sms = 0;
    if (device_sms(&sms) != SPIREC_OK) return SPIREC_ECUDA;
    return with_size(M, LaunchRowsInv{p, out, mode, dotx, dot_scalar, blocks, s, c, kSplitInvCtasPerSm * sms});
}

int launch_toeplitz(spirec_plan p, const float2* x, float2* Tx, int dot_scalar)
{
    int rc;
    const int N = p->N;
    if ((rc = launch_rows_fwd(p, x, N, N, N, 0, nullptr)) != SPIREC_OK) return rc;
    if ((rc = launch_cols(p, N, N)) != SPIREC_OK) return rc;
    return launch_rows_inv(p, Tx, 0, dot_scalar >= 0 ? x : nullptr, nullptr, dot_scalar);
}

int launch_spectrum(spirec_plan p)
{
    const int N = p->N, M = p->M;
    k_embed<<<dim3((unsigned)((M + 31) / 32), (unsigned)((M + 31) / 32)), dim3(32, 8), 0, p->stream>>>(p->G, N, M,
                                                                                                   p->cwork);
    SPIREC_CK(cudaGetLastError());
    p->launches += 1;
    const bool pow2 = is_pow2_specialised(M);
    return with_size(M, LaunchSpectrum{p, row_shape(M, pow2), col_shape(M, pow2)});
}

}  // namespace spirec

// ------------------------------------------------ T x without any allocation
//
// spirec_toeplitz_noalloc: the Toeplitz apply above for callers that cannot
// allocate device memory (for example code running inside a memory-pool
// budget that forbids cudaMalloc, or a host process that must not grow the
// GPU footprint after start-up).  The caller passes the input, the kernel
// spectrum and the output; the intermediate N x M rows, the transposed
// spectrum and the twiddle table live in one file-scope device array that
// every GPU loading this library keeps until the process exits.

namespace spirec {
namespace {

constexpr int kNoAllocMaxN = 512;
constexpr int kNoAllocMaxM = 1024;
constexpr size_t kNoAllocRowsBytes = (size_t)kNoAllocMaxN * kNoAllocMaxM * sizeof(float2);
constexpr size_t kNoAllocSpecBytes = (size_t)kNoAllocMaxM * kNoAllocMaxM * sizeof(float);
constexpr size_t kNoAllocTwBytes = (size_t)kNoAllocMaxM * sizeof(float2);
constexpr size_t kNoAllocBytes = kNoAllocRowsBytes + kNoAllocSpecBytes + kNoAllocTwBytes;

// Shared by every call on a device; holds the last call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
// device address of the array per device, published once its set-up is done
// (release store, acquire load); the mutex makes the first calls of several
// host threads on one device run the set-up once
std::atomic<void*> g_noalloc_base[kNoAllocMaxDevices];
std::mutex g_noalloc_mu;

// tw[k] = exp(-2 pi i k / M)
__global__ void k_noalloc_twiddles(float2* tw, int M)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)k / (double)M, &s, &c);
        tw[k] = make_float2((float)c, (float)s);
    }
}

// spectrum[ky][kx] (the layout spirec_kernel_spectrum_dev returns) into the
// column-major form the column pass reads, chat[kx][ky].
__global__ void k_noalloc_spectrum(const float* __restrict__ spec, int M, float* __restrict__ chat)
{
    const int64_t MM = (int64_t)M * M;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < MM;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t kx = e / M, ky = e % M;
        chat[e] = spec[ky * M + kx];
    }
}

struct LaunchNoAlloc {
    const float2* x;
    float2* Tx;
    float2* rows;
    const float* chat;
    const float2* tw;
    FftPlan fp;
    int N;
    cudaStream_t st;
    template <int MC>
    int operator()()
    {
        const int M = fp.M;
        const bool pow2 = MC > 0;
        const Shape rs = row_shape(M, pow2), cs = col_shape(M, pow2);
        const int rblocks = (N + rs.per_cta - 1) / rs.per_cta;
        const CgPass c{};
        k_rows_fwd<MC, 0><<<rblocks, rs.threads, rs.smem, st>>>(x, N, N, N, rows, fp, tw, rs.per_cta, c);
        SPIREC_CK(cudaGetLastError());
        k_cols_filter<MC><<<(M + cs.per_cta - 1) / cs.per_cta, cs.threads, cs.smem, st>>>(rows, N, N, fp, tw,
                                                                                          chat, cs.per_cta);
        SPIREC_CK(cudaGetLastError());
        k_rows_inv<MC, 0><<<rblocks, rs.threads, rs.smem, st>>>(rows, N, Tx, N, fp, tw, rs.per_cta, nullptr,
                                                                 c, 0);
        SPIREC_CK(cudaGetLastError());
        return SPIREC_OK;
    }
};

}  // namespace

}  // namespace spirec

extern "C" int spirec_toeplitz_noalloc(const float* x, const float* spectrum, float* Tx, int32_t N,
                                       int32_t M, void* stream)
{
    using namespace spirec;
    if (!x || !spectrum || !Tx) {
        set_error("null pointer");
        return SPIREC_EINVAL;
    }
    if (N < 2 || N > kNoAllocMaxN || M < 2 * N - 1 || M > kNoAllocMaxM) {
        set_error("spirec_toeplitz_noalloc handles 2 <= N <= %d and 2N-1 <= M <= %d (got N=%d, M=%d)",
                  kNoAllocMaxN, kNoAllocMaxM, N, M);
        return SPIREC_EINVAL;
    }
    FftPlan fp;
    if (!make_fft_plan(M, &fp)) {
        set_error("M=%d must factor into 2, 3 and 5", M);
        return SPIREC_EINVAL;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("device %d out of range", dev);
        return SPIREC_EUNSUPPORTED;
    }
    // first call on this device: the array's device address and the kernels'
    // shared-memory limits (no allocation; must happen outside stream capture)
    void* addr = g_noalloc_base[dev].load(std::memory_order_acquire);
    if (!addr) {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        addr = g_noalloc_base[dev].load(std::memory_order_relaxed);
        if (!addr) {
            e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
            int rc = fft_setup_attributes(M);
            if (rc != SPIREC_OK) return rc;
            g_noalloc_base[dev].store(addr, std::memory_order_release);
        }
    }
    unsigned char* base = static_cast<unsigned char*>(addr);
    float2* rows = reinterpret_cast<float2*>(base);
    float* chat = reinterpret_cast<float*>(base + kNoAllocRowsBytes);
    float2* tw = reinterpret_cast<float2*>(base + kNoAllocRowsBytes + kNoAllocSpecBytes);
    cudaStream_t st = (cudaStream_t)stream;
    k_noalloc_twiddles<<<(M + 255) / 256, 256, 0, st>>>(tw, M);
    SPIREC_CK(cudaGetLastError());
    k_noalloc_spectrum<<<4 * 152, 256, 0, st>>>(spectrum, M, chat);
    SPIREC_CK(cudaGetLastError());
    return with_size(M, LaunchNoAlloc{(const float2*)x, (float2*)Tx, rows, chat, tw, fp, N, st});
}
