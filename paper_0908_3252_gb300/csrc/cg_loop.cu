// cg_loop.cu -- the whole Polak-Ribiere loop (section 3.3 on the rewritten
// criterion of section 3.4) as ONE persistent cooperative kernel.
//
// One 512-thread block per SM (up to 128 registers a thread, so nothing
// spills: with the row caches in shared memory little L1 is left for local
// memory).  Block b owns the image rows [R0, R0 + RB) for the whole solve
// and keeps in shared memory f and d of those rows plus one halo row on each
// side, and T f - D, D, g and T d of its own rows.  Only the Toeplitz row buffers and one
// halo row of g per side pass through global memory (L2):
//   X   the row FFTs of g, overwritten by the column-filtered rows Y.
//
// One iteration, five grid synchronisations:
//   B  columns  column FFT * Chat * IFFT of X -> Y in X
//               [synchronisation without a value]
//   C  rows     row IFFTs of Y -> T g, and T d = -T g + beta T d_old (-T g on
//               a restart: T is linear, so the apply of the new direction
//               d = -g + beta d_old follows from the gradient's alone);
//               d = -g + beta d_old on the cached rows; sums
//               q1 = Re<d, 2 res>, q2 = Re<d, T d> and the penalty terms
//               of h'(0) and of the curvature at t = 0
//               [reduce 4 -> t1]
//   D, E        majorize-minimize steps of the line search at t1, t2, from
//               shared memory            [reduce 2 -> t2]  [reduce 2 -> t3]
//   A  update   f += t3 d, res += t3 T d, g = 2 res + grad R(f), the six
//               sums of J and beta; row FFTs of g -> X
//               [synchronisation; the six totals are formed during the next
//               column pass, which does not need beta, and J and beta at its
//               closing synchronisation]
// At M = 1024 every sequence the FFTs see is half zero (N <= 512 inputs of a
// 1024-point transform), so each 1024-point DFT splits exactly into two
// 512-point ones, X[2k + h] = DFT512(x w1024^(h n))[k], and one warp per
// half runs each as a register four-step (16 x 32): the row buffers hold a
// row as [h][k] (element 2k + h of the DFT at h * 512 + k), the column pass
// runs two warps per column, and the row passes two warps per row.
// An initial update without a step gives g(x0), J(x0) and beta = 0.  Every
// halo value is recomputed by the block that caches it from the same
// operands as its owner uses, so all copies of a pixel are bitwise equal.
//
// After each reduction one warp per value sums the per-block float-float
// partials (same order in every block) and every thread forms the line-search
// step from those totals in float-float arithmetic, so all blocks and threads
// hold the same step bit for bit.  The update's six sums are the exception: their partials are copied into shared
// memory during the next column pass and summed, with J and beta formed, at
// that pass's synchronisation (deferred_parts_fetch, deferred_parts_sum).
//
// Every grid synchronisation is a reduction over block partials behind an
// arrival counter (see grid_reduce).  Its wait is bounded in time (the
// launch's wait limit, 2 s unless a test sets it): on expiry the block raises
// an abort word and an error bit, every block returns at its next
// synchronisation, and the host reports SPIREC_ETIMEOUT.  No asynchronous
// copy is in flight at a synchronisation (the deferred partials are waited
// for before it), so a block that returns there leaves nothing behind.  The
// cooperative launch guarantees that all blocks are resident, so no wait
// depends on an unscheduled block.
#include <stdint.h>

#include <mutex>

#include "cg_device.cuh"
#include "fft_device.cuh"
#include "fft_reg.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace spirec {

namespace {

constexpr int kLoopThreads = 512;
constexpr int kMaxGroupsPerBlock = 8;
constexpr int kProf = 10;

struct LoopArgs {
    int N, iters, RB;  // RB: rows owned per block
    float2* f0;        // x0 in, the last iterate out
    float2* g;         // gradient rows (halo exchange)
    float2* res;       // T x0 - D in, T f - D out (the data term's residual)
    const float2* D;
    float2* X;
    const float* Chat;
    const float* ChatS;  // M = 1024: Chat in the split order of the column pass
    const float2* tw;
    FftPlan fp;
    Reg reg;
    double* scal;
    double* Jdev;
    float2* parts;     // block partials, P_NSLOTS x kMaxParts
    unsigned* counter;  // arrivals, zero at the launch
    unsigned* abort_word;
    int* err;
    unsigned long long wait_ns;  // limit of every grid wait (wait_limit_ns())
    int stall;                   // a test's injected stall (injected_stall())
};

// Loop scalars, one copy per block.  Thread 0 writes them (the reductions'
// totals: the warps that form them); every write is separated by a barrier
// from the reads of the same slot, and the line-search steps alternate
// between the two slots of tb.  The FP64 values are used by one thread only.
struct LoopShared {
    double red[8];  // grid sums of the deferred update reduction (and the first)
    FF redf[8];     // grid sums of the last grid_reduce
    float ws[32][8];  // warp sums of the block reduction in grid_reduce / grid_arrive_parts
    double ss, gg, J, beta;
    FF q1, q2, tb[2];  // line-search scalars, float-float: they sit on the critical path
    float beta_f;
    int restart, ok;
    unsigned long long prof[kProf], tmark;
};

template <int MC>
struct Geo {
    static constexpr int RPC = 4 * kLoopThreads / MC;  // rows per FFT group: RPC * MC = 4 * threads
    static constexpr int CBPT = MC >= 256 ? 2 : 1;     // column groups: CBPT butterflies per thread
    static constexpr int CPC = CBPT * RPC;
    // the wide column group (twice the butterflies per thread), when it fits
    static constexpr int CBPT2 = CBPT;  // (wider column groups spill registers)
    static constexpr int CPC2 = CBPT2 * RPC;
    static constexpr int LDR = fftd::seq_len<MC>(MC);
    static constexpr int LDC = LDR + 4;
    // M = 1024: the split 512-point FFTs (fwd512 / inv512), two warps per
    // sequence; the column pass takes FS_COLS columns per group, each
    // column's shared-memory area LDF long: the column itself, then the two
    // warps' exchange areas of WA each (LDF = 2 mod 16 keeps the staging
    // stores of 8 neighbouring columns on distinct banks)
    static constexpr bool FOURSTEP = MC == 1024;
    static constexpr int FS_COLS = 8;
    static constexpr int WA = 544;  // 16 x 33 (forward), 32 x 17 (inverse)
    static constexpr int LDF = 1090;
    static constexpr int FB_ROWS = FOURSTEP ? 16 * WA : 2 * RPC * LDR;
    static constexpr int FB_COLS = FOURSTEP ? FS_COLS * LDF : CPC2 * LDC;
    static constexpr int FBUF = FB_ROWS > FB_COLS ? FB_ROWS : FB_COLS;
    // staged radix-4 twiddles (not at M = 1024), then (M = 1024) the tables
    // T16[k2][l] = w512^(l k2) and WN[j][l] = w1024^(l + 32 j)
    static constexpr int TW_R4 = FOURSTEP ? 0 : (fftd::staged_twiddles_size(MC) + 1) & ~1;  // 16-byte aligned
    static constexpr int TW = TW_R4 + (FOURSTEP ? 1024 : 0);
};

// dynamic shared memory of a block owning RB rows of an N-wide image: the
// FFT buffer, the staged twiddle table, the row caches
template <int MC>
size_t loop_smem(int N, int RB)
{
    const size_t grid = (size_t)((N + RB - 1) / RB);
    // FFT buffer, twiddles, f and d of RB + 2 rows, T f - D, D, g, T d of RB rows,
    // and the deferred update partials (kUpdVals x even (grid + 1), and one
    // float2 to align them to 16 bytes)
    return ((size_t)Geo<MC>::FBUF + Geo<MC>::TW + (size_t)(2 * (RB + 2) + 4 * RB) * N +
            kUpdVals * ((grid + 2) & ~(size_t)1) + 2) * sizeof(float2);
}

__device__ __forceinline__ uint64_t gtimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------ grid-wide reductions
//
// A grid synchronisation is a reduction: warp k of every block writes the
// block's float-float partial of value k, and thread 0, after a named barrier
// of those warps, adds one to an arrival counter with a release reduction
// (no return value awaited) and polls the counter with
// acquire loads until all blocks of this synchronisation have arrived (the
// counter grows monotonically during a launch: the n-th synchronisation
// waits for n * gridDim.x).  Then one warp per value sums the partials of
// all blocks in index order.

__device__ __forceinline__ bool grid_arrive_wait(unsigned* counter, unsigned target, unsigned* abort_word, int* err,
                                                 unsigned long long limit_ns)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(counter) : "memory");
    const uint64_t t0 = gtimer();
    for (unsigned spins = 1;; ++spins) {
        unsigned cur;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(counter) : "memory");
        if ((int)(cur - target) >= 0) return true;
        if ((spins & 15) == 0) {
            unsigned ab;
            asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(ab) : "l"(abort_word) : "memory");
            if (ab) return false;
            if (gtimer() - t0 > limit_ns) {
                atomicExch(abort_word, 1u);
                atomicOr(err, E_TIMEOUT);
                return false;
            }
        }
    }
}

// The block's partials of K values to slot `slot` and the arrival: each
// warp sums its lanes in FP32, then warp k sums value k over the warps in
// float-float (the trees of block_partial) and stores it; thread 0 arrives
// after a named barrier of those warps (its release covers their stores) and
// waits.  S.ws is read only between this call's first and last barriers.
template <int K>
__device__ __forceinline__ void block_publish(float (&v)[K], float2* parts, int slot, unsigned seq, LoopShared& S,
                                              unsigned* counter, unsigned* abort_word, int* err,
                                              unsigned long long limit_ns)
{
    static_assert(K >= 1 && K <= 8, "one warp per value");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) S.ws[warp][k] = v[k];
    __syncthreads();
    if (warp < K) {
        const int nw = (blockDim.x + 31) >> 5;
        const FF bt = warp_sum_ff(FF{lane < nw ? S.ws[lane][warp] : 0.f, 0.f});
        if (lane == 0) parts[(slot + warp) * kMaxParts + blockIdx.x] = make_float2(bt.hi, bt.lo);
        if constexpr (K > 1) asm volatile("bar.sync 2, %0;" ::"r"(32 * K) : "memory");
        if (threadIdx.x == 0) S.ok = grid_arrive_wait(counter, seq * gridDim.x, abort_word, err, limit_ns) ? 1 : 0;
    }
    __syncthreads();
}

// Block partials of K values to slot `slot`, the synchronisation, then the
// grid totals as float-float pairs in S.redf, readable by every thread on
// return.  seq counts the synchronisations of the launch (the same in every
// thread).
template <int K>
__device__ __forceinline__ bool grid_reduce(float (&v)[K], float2* parts, int slot, unsigned& seq, LoopShared& S,
                                            unsigned* counter, unsigned* abort_word, int* err,
                                            unsigned long long limit_ns)
{
    ++seq;
    block_publish<K>(v, parts, slot, seq, S, counter, abort_word, err, limit_ns);
    if (!S.ok) return false;
    const int warp = threadIdx.x >> 5;
    if (warp < K) {
        const FF a = warp_sum_parts(parts + (slot + warp) * kMaxParts, gridDim.x);
        if ((threadIdx.x & 31) == 0) S.redf[warp] = a;
    }
    __syncthreads();
    return true;
}

// The first half of grid_reduce: the block partials to slot `slot` and the
// synchronisation; the totals are formed later (deferred_parts_fetch /
// deferred_parts_sum), off the critical path.
template <int K>
__device__ __forceinline__ bool grid_arrive_parts(float (&v)[K], float2* parts, int slot, unsigned& seq,
                                                  LoopShared& S, unsigned* counter, unsigned* abort_word, int* err,
                                                  unsigned long long limit_ns)
{
    ++seq;
    block_publish<K>(v, parts, slot, seq, S, counter, abort_word, err, limit_ns);
    return S.ok != 0;
}

// Copies the K x gridDim.x partials of a past synchronisation into shared
// memory by asynchronous 16-byte copies through L2 (cp.async.cg: no register
// and no L1 line, so later rounds never see stale data); the block goes on
// with other work and waits for them in deferred_parts_sum.
template <int K>
__device__ __forceinline__ void deferred_parts_fetch(const float2* parts, int slot, float2* pbuf)
{
    const int nch = (gridDim.x + 1) >> 1;  // 16-byte chunks of a value (two partials each)
    for (int e = threadIdx.x; e < K * nch; e += blockDim.x) {
        const int k = e / nch, c = e - k * nch;
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(pbuf + k * 2 * nch + 2 * c);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst),
                     "l"(parts + (slot + k) * kMaxParts + 2 * c)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Waits for deferred_parts_fetch's copies; warps 1..K sum value k = warp - 1
// of the block partials in index order (as warp_sum_parts) into S.red.
// Contains __syncthreads() and a named barrier over warps 1..K+1 (K + 1 <= 15).
template <int K>
__device__ __forceinline__ void deferred_parts_sum(const float2* pbuf, LoopShared& S)
{
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nch = (gridDim.x + 1) >> 1;
    if (warp >= 1 && warp <= K) {
        const float2* v = pbuf + (warp - 1) * 2 * nch;
        FF acc{0.f, 0.f};
        for (int i = lane; i < (int)gridDim.x; i += 32) acc = ff_add(acc, FF{v[i].x, v[i].y});
        acc = warp_sum_ff(acc);
        if (lane == 0) S.red[warp - 1] = ff_to_double(acc);
    }
}

// J and beta from the update sums in S.red (one thread): J(f_k), the PR+
// beta of the next direction (0: restart), J_hist[k] by block 0.
__device__ __forceinline__ void finish_update(const LoopArgs& A, LoopShared& S, int k)
{
    double J, beta_n;
    cgd::update_finish(S.red, S.ss, S.gg, false, &J, &beta_n);
    S.gg = S.red[0];
    S.J = J;
    S.beta = beta_n;
    S.beta_f = (float)beta_n;
    S.restart = beta_n == 0.0;
    if (blockIdx.x == 0) A.Jdev[k] = J;
}

// partial slots: consecutive synchronisations use different slots (a fast
// block may write the next partials while a slow one still reads these), and
// a slot's next use is at least two synchronisations later
constexpr int L_A = 0;   // 6
constexpr int L_C = 6;   // 4
constexpr int L_D = 10;  // 2
constexpr int L_E = 12;  // 2

// The rows one block works on: own rows [R0, R0 + nown), cached rows
// [hlo, hhi] (the own rows and the existing halo rows).
struct Rows {
    int N, R0, nown, hlo, hhi;
    __device__ __forceinline__ int cache(int r) const { return (r - R0 + 1) * N; }  // row offset in cf, cd
};

// (row, column) of the first element of a per-pixel loop over rows of N
// pixels that starts at threadIdx.x, and of the next one when it strides by
// the block size (one division a loop, none a pixel).
__device__ __forceinline__ int first_row(int N) { return (int)threadIdx.x / N; }
__device__ __forceinline__ int first_col(int N) { return (int)threadIdx.x - first_row(N) * N; }
__device__ __forceinline__ void step_pixel(int& q, int& m, int N)
{
    m += kLoopThreads;
    while (m >= N) {
        m -= N;
        ++q;
    }
}

// ------------------------------------------------- split FFTs, M = 1024

// x[i] = row[i] + row[i + 16] (lanes 0-15) or (row[i] - row[i + 16]) w32^i
// (lanes 16-31), i < 16.
template <int I = 0>
__device__ __forceinline__ void halves_fwd(float2 (&x)[16], const float2* row, bool half)
{
    if constexpr (I < 16) {
        const float2 u = row[I], v = row[I + 16];
        x[I] = half ? freg::mulw<false, I>(freg::sub(u, v)) : freg::add(u, v);
        halves_fwd<I + 1>(x, row, half);
    }
}

// out[i] = x[i] (lanes 0-15) or x[i] w32^-i (lanes 16-31), i < 16.
template <int I = 0>
__device__ __forceinline__ void store_odd_twiddled(const float2 (&x)[16], float2* out, bool half)
{
    if constexpr (I < 16) {
        out[I] = half ? freg::mulw<true, I>(x[I]) : x[I];
        store_odd_twiddled<I + 1>(x, out, half);
    }
}

// One warp, the 512-point DFT of the sequence whose element lane + 32 j is in
// x[j] (j < 16): a 16-point DFT over the registers, twiddles w512^(lane k2),
// an exchange through this warp's area (16 x 33), a radix-2 step across the
// lane halves (lane = k2 + 16 half: half 0 adds the two halves of the
// exchanged row k2, half 1 subtracts and twiddles by w32^i), and a 16-point
// DFT over the registers.  Element lane + 32 q of the result ends in
// x[bitrev4(q)].  t16[k2 * 32 + l] = w512^(l k2).
__device__ __forceinline__ void fwd512(float2 (&x)[16], float2* area, const float2* t16, int lane)
{
    freg::dft16_dif<false>(x);
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) area[k2 * 33 + lane] = cmul(x[freg::bitrev4(k2)], t16[k2 * 32 + lane]);
    __syncwarp();
    halves_fwd(x, area + (lane & 15) * 33, lane >= 16);
    __syncwarp();
    freg::dft16_dif<false>(x);
}

// One warp, u[n] = sum_k Z[k] w512^(-n k) for Z[lane + 32 q] in x[bitrev4(q)]
// (the order fwd512 leaves): a 16-point inverse DFT over the registers gives,
// per lane = k2 + 16 half, the inverse DFT over the even (half 0) or odd
// (half 1, then times w32^-i) k1 of the k = k2 + 16 k1 with this k2; the two
// combine through the area (32 x 17) into the 32-point inverse DFT over k1,
// lane n1 takes its values for every k2, twiddles by w512^(-n1 k2) and runs
// a 16-point inverse DFT over the registers.  u[lane + 32 n2] ends in
// x[bitrev4(n2)].
__device__ __forceinline__ void inv512(float2 (&x)[16], float2* area, const float2* t16, int lane)
{
    freg::dft16_dit<true>(x);
    const bool half = lane >= 16;
    store_odd_twiddled(x, area + lane * 17, half);
    __syncwarp();
    const int i = lane & 15;
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) {
        const float2 e = area[k2 * 17 + i], o = area[(16 + k2) * 17 + i];
        x[k2] = cmul(half ? freg::sub(e, o) : freg::add(e, o), conjf2(t16[k2 * 32 + lane]));
    }
    __syncwarp();
    freg::dft16_dif<true>(x);
}

// Columns [x0, x0 + 8) of the M = 1024 Toeplitz pass, two warps per column
// (warp 2 cc + h: column cc, output parity h).  The block loads the 8
// columns of X (row FFTs of g) as 64-byte row pieces and parks them in
// shared memory.  Warp (cc, h) takes x[n] w1024^(h n) of its
// column (n = lane + 32 j < 512; rows >= n_in are zero), runs fwd512 (the
// column spectrum at ky = 2 k + h), multiplies by the spectrum, runs inv512,
// and multiplies by w1024^(-h n); the two warps' results add up to the
// filtered column, whose rows < n_in go back to X.  chs holds the spectrum in
// this split order: chs[c * 1024 + h * 512 + k] = Chat[kx(c)][2 k + h].
// wn[j * 32 + l] = w1024^(l + 32 j).
template <typename F>
__device__ __forceinline__ void cols_split(float2* X, int n_in, int x0, const float* __restrict__ chs,
                                           const float2* t16, const float2* wn, float2* fbuf, F&& after_staging)
{
    constexpr int M = 1024, COLS = 8, LDF = 1090, WA = 544;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cc = warp >> 1, h = warp & 1;
    {
        // 8 columns x 512 rows (rows >= n_in are zero), 8 per thread
        float2 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int e = tid + i * kLoopThreads;
            const int y = e >> 3;
            v[i] = y < n_in ? __ldcg(X + (int64_t)y * M + x0 + (e & 7)) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int e = tid + i * kLoopThreads;
            fbuf[(e & 7) * LDF + (e >> 3)] = v[i];
        }
    }
    __syncthreads();
    after_staging();  // work that should not compete with the staging loads
    // the spectrum values of this warp (used after the forward FFT)
    float hs[16];
    {
        const float* ch = chs + (int64_t)(x0 + cc) * M + h * 512 + lane;
#pragma unroll
        for (int q = 0; q < 16; ++q) hs[q] = __ldcg(ch + 32 * q);
    }
    float2 x[16];
    {
        const float2* col = fbuf + cc * LDF + lane;
#pragma unroll
        for (int j = 0; j < 16; ++j) x[j] = h ? cmul(col[32 * j], wn[j * 32 + lane]) : col[32 * j];
    }
    // the column is in both warps' registers: warp 0's exchange area, which
    // overlaps the staged column (warp 1's lies past it), may be overwritten
    // once the pair has passed (named barrier 8 + cc)
    asm volatile("bar.sync %0, 64;" ::"r"(8 + cc) : "memory");
    float2* area = fbuf + cc * LDF + h * WA;
    fwd512(x, area, t16, lane);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        float2& r = x[freg::bitrev4(q)];
        r = make_float2(r.x * hs[q], r.y * hs[q]);
    }
    inv512(x, area, t16, lane);
    // y[n] = u_0[n] + w1024^(-n) u_1[n] (n = lane + 32 n2), the two warps of
    // the column a half each: warp 0 the rows n < 256, warp 1 the rest.  Each
    // first hands the other its half of the operands (warp 1 through its
    // area, warp 0 through the column's upper half), then a barrier of the
    // pair (named barrier 8 + cc)
    float2* col = fbuf + cc * LDF;
    float2* a1 = fbuf + cc * LDF + WA;
    if (h) {
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) a1[lane + 32 * n2] = cmul(x[freg::bitrev4(n2)], conjf2(wn[n2 * 32 + lane]));
    } else {
#pragma unroll
        for (int n2 = 8; n2 < 16; ++n2) col[lane + 32 * n2] = x[freg::bitrev4(n2)];
    }
    asm volatile("bar.sync %0, 64;" ::"r"(8 + cc) : "memory");
    if (h) {
#pragma unroll
        for (int n2 = 8; n2 < 16; ++n2) {
            const int n = lane + 32 * n2;
            col[n] = freg::add(col[n], cmul(x[freg::bitrev4(n2)], conjf2(wn[n2 * 32 + lane])));
        }
    } else {
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) col[lane + 32 * n2] = freg::add(x[freg::bitrev4(n2)], a1[lane + 32 * n2]);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int e = tid + i * kLoopThreads;
        const int y = e >> 3, c = e & 7;
        if (y < n_in) X[(int64_t)y * M + x0 + c] = fbuf[c * LDF + y];
    }
    (void)COLS;
}

// Two warps per row (warp 2 q + h), the split row FFTs at M = 1024 of rows
// [g0, g0 + 8) of the own-row cache src (N values a row, zero beyond):
// X[row][h * 512 + k] = DFT1024(src row)[2 k + h].
__device__ __forceinline__ void rows_fwd_split(const float2* src, int N, int nrows, float2* Xrows, float2* fbuf,
                                               const float2* t16, const float2* wn)
{
    constexpr int M = 1024, WA = 544;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = warp >> 1, h = warp & 1;
    if (q < nrows) {
        float2 x[16];
        const float2* r = src + q * N;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int m = lane + 32 * j;
            const float2 v = m < N ? r[m] : make_float2(0.f, 0.f);
            x[j] = h ? cmul(v, wn[j * 32 + lane]) : v;
        }
        fwd512(x, fbuf + warp * WA, t16, lane);
        float2* out = Xrows + (int64_t)q * M + h * 512 + lane;
#pragma unroll
        for (int q2 = 0; q2 < 16; ++q2) out[32 * q2] = x[freg::bitrev4(q2)];
    }
}

// ---------------------------------------------------------------- phase A

// Gradient of every own pixel (phi fixed at compile time): g into the
// own-row cache and global memory (the halo rows of the neighbours), and the
// six update sums of cgd::update_pixel.
template <int KIND, bool FIRST>
__device__ __forceinline__ void grad_rows(const LoopArgs& A, const Rows& R, const float2* cf, const float2* cd,
                                          const float2* cRes, const float2* cD, float2* cg, float (&a)[kUpdVals])
{
    const int N = R.N;
    const Reg reg = A.reg;
    for (int e = threadIdx.x, oq = first_row(N), m = first_col(N); e < R.nown * N; e += kLoopThreads, step_pixel(oq, m, N)) {
        const int n = R.R0 + oq;
        const bool has_u = n > 0, has_l = m > 0, has_d = n + 1 < N, has_r = m + 1 < N;
        const float2* row = cf + R.cache(n);
        const float2 fc = row[m];
        const float2 fu = has_u ? row[m - N] : fc, fdn = has_d ? row[m + N] : fc;
        const float2 fl = has_l ? row[m - 1] : fc, fr = has_r ? row[m + 1] : fc;
        const float2 rs = cRes[e], dv = cD[e];
        float rv;
        const float2 gp = cgd::grad_at<KIND>(fc, fu, fl, fdn, fr, rs, has_u, has_l, has_d, has_r, reg, rv);
        a[0] += cgd::redot(gp, gp);
        if (!FIRST) {
            a[1] += cgd::redot(gp, cg[e]);
            a[2] += cgd::redot(gp, cd[R.cache(n) + m]);
        }
        a[3] += rv;
        a[4] += cgd::redot(fc, dv);
        a[5] += cgd::redot(fc, rs);
        cg[e] = gp;
        A.g[(int64_t)n * N + m] = gp;
    }
}

// One penalty term of the line search from the precomputed quantities of its
// edge (or pixel) z, w: |z|^2, Re(conj(z) w), |w|^2.  |z + t w|^2 = az + 2 t
// bzw + t^2 cw; num += lambda b(|z + t w|) (bzw + t cw), den += lambda b cw.
// A missing edge has all three zero and adds nothing.
template <int KIND>
__device__ __forceinline__ void ls_edge(float lam, float alpha, int kind, float az, float bzw, float cw, float t,
                                        float& num, float& den)
{
    const float x2 = fmaxf(fmaf(t, fmaf(t, cw, 2.f * bzw), az), 0.f);
    const float b = lam * phi_weight_k<KIND>(kind, alpha, x2);
    num = fmaf(b, fmaf(t, cw, bzw), num);
    den = fmaf(b, cw, den);
}

// Line-search sums of the own pixels at step t (phi fixed at compile time).
// T0 (the first step, t = 0): also Re<d, 2 (T f - D)> into acc[0] and
// Re<d, T d> into acc[3], the penalty terms into acc[1], acc[2]; with PRE it
// stores each edge's |z|^2, Re(conj(z) w), |w|^2 (z of f, w of d) in the
// planes E (plane k at E + k nown N: right edge 0-2, down edge 3-5, pixel
// 6-8 when lambda0 != 0).  Later steps (!T0) with PRE read the planes
// instead of f and d.
template <int KIND, bool T0, bool PRE>
__device__ __forceinline__ void ls_rows(const Reg& reg, const Rows& R, const float2* cf, const float2* cd,
                                        const float2* cRes, const float2* cD, const float2* cTd, float t,
                                        float* acc, float* E)
{
    const int N = R.N, P = R.nown * N;
    const bool l1 = reg.lambda1 != 0.f, l0 = reg.lambda0 != 0.f;
    for (int e = threadIdx.x, q = first_row(N), m = first_col(N); e < P; e += kLoopThreads, step_pixel(q, m, N)) {
        if constexpr (PRE && !T0) {
            if (l1) {
                ls_edge<KIND>(reg.lambda1, reg.alpha1, reg.kind, E[e], E[P + e], E[2 * P + e], t, acc[0], acc[1]);
                ls_edge<KIND>(reg.lambda1, reg.alpha1, reg.kind, E[3 * P + e], E[4 * P + e], E[5 * P + e], t, acc[0],
                              acc[1]);
            }
            if (l0)
                ls_edge<KIND>(reg.lambda0, reg.alpha0, reg.kind, E[6 * P + e], E[7 * P + e], E[8 * P + e], t, acc[0],
                              acc[1]);
        } else {
            const int n = R.R0 + q;
            const bool has_r = m + 1 < N, has_d = n + 1 < N;
            const float2* fr0 = cf + R.cache(n);
            const float2* dr0 = cd + R.cache(n);
            const float2 fp = fr0[m], dp = dr0[m];
            const float2 fr = has_r ? fr0[m + 1] : fp, dr = has_r ? dr0[m + 1] : dp;
            const float2 fd = has_d ? fr0[m + N] : fp, dd = has_d ? dr0[m + N] : dp;
            float* num = T0 ? &acc[1] : &acc[0];
            float* den = T0 ? &acc[2] : &acc[1];
            if constexpr (T0) {
                acc[0] += 2.f * cgd::redot(dp, cRes[e]);
                acc[3] += cgd::redot(dp, cTd[e]);
            }
            if constexpr (PRE) {
                // (masked neighbours carry the centre value: z = w = 0)
                if (l1) {
                    const float2 zr = cgd::f2sub(fr, fp), wr = cgd::f2sub(dr, dp);
                    const float2 zd = cgd::f2sub(fd, fp), wd = cgd::f2sub(dd, dp);
                    const float a0 = cgd::redot(zr, zr), b0 = cgd::redot(zr, wr), c0 = cgd::redot(wr, wr);
                    const float a1 = cgd::redot(zd, zd), b1 = cgd::redot(zd, wd), c1 = cgd::redot(wd, wd);
                    E[e] = a0;
                    E[P + e] = b0;
                    E[2 * P + e] = c0;
                    E[3 * P + e] = a1;
                    E[4 * P + e] = b1;
                    E[5 * P + e] = c1;
                    ls_edge<KIND>(reg.lambda1, reg.alpha1, reg.kind, a0, b0, c0, t, *num, *den);
                    ls_edge<KIND>(reg.lambda1, reg.alpha1, reg.kind, a1, b1, c1, t, *num, *den);
                }
                if (l0) {
                    const float a2 = cgd::redot(fp, fp), b2 = cgd::redot(fp, dp), c2 = cgd::redot(dp, dp);
                    E[6 * P + e] = a2;
                    E[7 * P + e] = b2;
                    E[8 * P + e] = c2;
                    ls_edge<KIND>(reg.lambda0, reg.alpha0, reg.kind, a2, b2, c2, t, *num, *den);
                }
            } else {
                cgd::ls_terms<KIND>(fp, dp, fr, dr, fd, dd, has_r, has_d, reg, t, *num, *den);
            }
        }
    }
}

// Whether the line-search planes of a block fit in its FFT buffer (free from
// the row pass to the update): 6 or 9 floats a pixel.
__device__ __forceinline__ bool ls_planes_fit(const Reg& reg, int npix, int fbuf_float2)
{
    const int planes = reg.lambda0 != 0.f ? 9 : 6;
    return planes * npix <= 2 * fbuf_float2;
}

// The per-pixel loops above for the run-time phi.
template <bool FIRST>
__device__ __forceinline__ void grad_rows_any(const LoopArgs& A, const Rows& R, const float2* cf, const float2* cd,
                                              const float2* cRes, const float2* cD, float2* cg, float (&a)[kUpdVals])
{
    switch (A.reg.kind) {
    case SPIREC_PHI_HUBER: grad_rows<SPIREC_PHI_HUBER, FIRST>(A, R, cf, cd, cRes, cD, cg, a); break;
    case SPIREC_PHI_HYPERBOLIC: grad_rows<SPIREC_PHI_HYPERBOLIC, FIRST>(A, R, cf, cd, cRes, cD, cg, a); break;
    default: grad_rows<SPIREC_PHI_QUADRATIC, FIRST>(A, R, cf, cd, cRes, cD, cg, a); break;
    }
}

template <bool T0, bool PRE>
__device__ __forceinline__ void ls_rows_k(const Reg& reg, const Rows& R, const float2* cf, const float2* cd,
                                          const float2* cRes, const float2* cD, const float2* cTd, float t, float* acc,
                                          float* E)
{
    switch (reg.kind) {
    case SPIREC_PHI_HUBER: ls_rows<SPIREC_PHI_HUBER, T0, PRE>(reg, R, cf, cd, cRes, cD, cTd, t, acc, E); break;
    case SPIREC_PHI_HYPERBOLIC:
        ls_rows<SPIREC_PHI_HYPERBOLIC, T0, PRE>(reg, R, cf, cd, cRes, cD, cTd, t, acc, E);
        break;
    default: ls_rows<SPIREC_PHI_QUADRATIC, T0, PRE>(reg, R, cf, cd, cRes, cD, cTd, t, acc, E); break;
    }
}

template <bool T0>
__device__ __forceinline__ void ls_rows_any(const Reg& reg, const Rows& R, const float2* cf, const float2* cd,
                                            const float2* cRes, const float2* cD, const float2* cTd, float t,
                                            float* acc, float* E, bool pre)
{
    if (pre)
        ls_rows_k<T0, true>(reg, R, cf, cd, cRes, cD, cTd, t, acc, E);
    else
        ls_rows_k<T0, false>(reg, R, cf, cd, cRes, cD, cTd, t, acc, E);
}

// Step (unless FIRST), gradient and the six update sums over the own rows
// (the sums of cgd::update_pixel); with do_fft the row FFTs of g go to X.
// Rows go through the FFT RX * RPC at a time (RX butterflies per thread).
template <int MC, bool FIRST, int RX>
__device__ __forceinline__ void phase_update(const LoopArgs& A, const Rows& R, float2* fbuf, const float2* stw,
                                             float2* cf,
                                             const float2* cd, float2* cRes, const float2* cD, float2* cg,
                                             const float2* cTd, float t, bool do_fft, float (&a)[kUpdVals])
{
    using G = Geo<MC>;
    const int N = R.N;
    if (!FIRST) {
        const int nc = (R.hhi - R.hlo + 1) * N;
        float2* fr0 = cf + R.cache(R.hlo);
        const float2* dr0 = cd + R.cache(R.hlo);
        for (int e = threadIdx.x; e < nc; e += kLoopThreads) fr0[e] = cgd::f2axpy(t, dr0[e], fr0[e]);
        for (int e = threadIdx.x; e < R.nown * N; e += kLoopThreads) cRes[e] = cgd::f2axpy(t, cTd[e], cRes[e]);
        __syncthreads();
    }
    if constexpr (G::FOURSTEP) {
        // gradient of every own pixel, then the split row FFTs of g, two
        // warps a row, eight rows at a time
        grad_rows_any<FIRST>(A, R, cf, cd, cRes, cD, cg, a);
        if (do_fft) {
            __syncthreads();  // g of every own row is in cg
            for (int g0 = 0; g0 < R.nown; g0 += 8)
                rows_fwd_split(cg + g0 * N, N, min(8, R.nown - g0), A.X + (int64_t)(R.R0 + g0) * MC, fbuf, stw,
                               stw + 512);
        }
    } else {
        // gradient of every own pixel, then the row FFTs of g, RX * RPC rows
        // at a time
        grad_rows_any<FIRST>(A, R, cf, cd, cRes, cD, cg, a);
        if (do_fft) {
            __syncthreads();  // g of every own row is in cg
            for (int g0 = 0; g0 < R.nown; g0 += RX * G::RPC) {
                const int nr = min(RX * G::RPC, R.nown - g0);
#pragma unroll
                for (int i = 0; i < 4 * RX; ++i) {
                    const int e = threadIdx.x + i * kLoopThreads;
                    const int q = e / MC, m = e - q * MC;
                    fbuf[q * G::LDR + fftd::sidx<MC>(m)] = q < nr && m < N ? cg[(g0 + q) * N + m] : make_float2(0.f, 0.f);
                }
                __syncthreads();
                fftd::fft_pow2<MC, false, RX, true>(fbuf, G::LDR, stw);
#pragma unroll
                for (int i = 0; i < 4 * RX; ++i) {
                    const int e = threadIdx.x + i * kLoopThreads;
                    const int q = e / MC, m = e - q * MC;
                    if (q < nr) A.X[(int64_t)(R.R0 + g0 + q) * MC + m] = fbuf[q * G::LDR + fftd::sidx<MC>(m)];
                }
                __syncthreads();
            }
        }
    }
}

// ---------------------------------------------------------------- phase C

// d = -g + beta d_old on the cached rows, by the nthr threads tid = 0 ..
// nthr - 1 (N <= 2 nthr: 256 threads at M = 1024, where N <= 512, and 512
// threads up to N = 1024).  The halo rows' g comes from their owners via L2:
// those loads go first, so their latency overlaps the own rows.
__device__ __forceinline__ void direction_rows(const float2* gglob, const Rows& R, float2* cd, const float2* cg,
                                               float beta, bool restart, int tid, int nthr)
{
    const int N = R.N;
    const bool up = R.hlo < R.R0, dn = R.hhi >= R.R0 + R.nown;
    constexpr int KH = 2;
    float2 hu[KH], hd[KH];
#pragma unroll
    for (int k = 0; k < KH; ++k) {
        const int m = tid + k * nthr;
        hu[k] = up && m < N ? __ldcg(gglob + (int64_t)R.hlo * N + m) : make_float2(0.f, 0.f);
        hd[k] = dn && m < N ? __ldcg(gglob + (int64_t)R.hhi * N + m) : make_float2(0.f, 0.f);
    }
    float2* own = cd + R.cache(R.R0);
    for (int e = tid; e < R.nown * N; e += nthr) own[e] = fftd::new_direction(cg[e], own[e], beta, restart);
#pragma unroll
    for (int k = 0; k < KH; ++k) {
        const int m = tid + k * nthr;
        if (m < N) {
            if (up) {
                float2& v = cd[R.cache(R.hlo) + m];
                v = fftd::new_direction(hu[k], v, beta, restart);
            }
            if (dn) {
                float2& v = cd[R.cache(R.hhi) + m];
                v = fftd::new_direction(hd[k], v, beta, restart);
            }
        }
    }
}

// Row IFFTs of Y (in X) -> T d of the own rows, RX * RPC rows at a time; the
// new direction on every cached row (at M = 1024 with at most four own rows,
// by the eight warps the row IFFTs leave idle, meanwhile); the four sums of
// the first line-search step.
template <int MC, int RX>
__device__ __forceinline__ void phase_rows(const LoopArgs& A, const Rows& R, float2* fbuf, const float2* stw,
                                           const float2* cf,
                                           float2* cd, const float2* cRes, const float2* cD, const float2* cg,
                                           float2* cTd, float beta, bool restart, float (&acc)[4])
{
    using G = Geo<MC>;
    const int N = R.N;
    const bool dir_aside = G::FOURSTEP && R.nown <= 4;  // warps 8 .. 15 have no row to transform
    if constexpr (G::FOURSTEP) {
        // the split row IFFTs of Y, two warps a row (warp 2 q + h takes the
        // elements 2 k + h), eight rows at a time: T g = u_0 + w1024^(-m) u_1
        // on the columns m < N
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int h = warp & 1;
        float2* area = fbuf + warp * G::WA;
        for (int g0 = 0; g0 < R.nown; g0 += 8) {
            const int q = g0 + (warp >> 1);
            const bool active = q < R.nown;
            float2 x[16];
            if (active) {
                const float2* yr = A.X + (int64_t)(R.R0 + q) * MC + h * 512 + lane;
#pragma unroll
                for (int q2 = 0; q2 < 16; ++q2) x[freg::bitrev4(q2)] = __ldcg(yr + 32 * q2);
                inv512(x, area, stw, lane);
                // T g[m] = u_0[m] + w1024^(-m) u_1[m], the row's two warps a
                // half each (warp 0 the columns m < 256), after handing each
                // other their halves of the operands and a barrier of the pair
                const float2* wn = stw + 512;
                float2* a0 = fbuf + (warp & ~1) * G::WA;
                float2* a1 = a0 + G::WA;
                if (h) {
#pragma unroll
                    for (int n2 = 0; n2 < 8; ++n2)
                        a1[lane + 32 * n2] = cmul(x[freg::bitrev4(n2)], conjf2(wn[n2 * 32 + lane]));
                } else {
#pragma unroll
                    for (int n2 = 8; n2 < 16; ++n2) a0[lane + 32 * n2] = x[freg::bitrev4(n2)];
                }
                asm volatile("bar.sync %0, 64;" ::"r"(8 + (warp >> 1)) : "memory");
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int n2 = h ? 8 + i : i;
                    const int m = lane + 32 * n2;
                    if (m < N) {
                        const float2 tg = h ? freg::add(a0[m], cmul(x[freg::bitrev4(n2)], conjf2(wn[n2 * 32 + lane])))
                                            : freg::add(x[freg::bitrev4(n2)], a1[m]);
                        float2& td = cTd[q * N + m];
                        td = fftd::new_direction(tg, td, beta, restart);
                    }
                }
            } else if (dir_aside && warp >= 8) {
                direction_rows(A.g, R, cd, cg, beta, restart, (int)threadIdx.x - 256, kLoopThreads - 256);
            }
            __syncthreads();
        }
    }
    for (int g0 = 0; g0 < (G::FOURSTEP ? 0 : R.nown); g0 += RX * G::RPC) {
        const int nr = min(RX * G::RPC, R.nown - g0);
        float2 v[4 * RX];
#pragma unroll
        for (int i = 0; i < 4 * RX; ++i) {
            const int e = threadIdx.x + i * kLoopThreads;
            const int q = e / MC, m = e - q * MC;
            v[i] = q < nr ? __ldcg(A.X + (int64_t)(R.R0 + g0 + q) * MC + m) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < 4 * RX; ++i) {
            const int e = threadIdx.x + i * kLoopThreads;
            const int q = e / MC, m = e - q * MC;
            fbuf[q * G::LDR + fftd::sidx<MC>(m)] = v[i];
        }
        __syncthreads();
        fftd::fft_pow2<MC, true, RX, true>(fbuf, G::LDR, stw);
        for (int e = threadIdx.x; e < nr * N; e += kLoopThreads) {
            const int q = e / N, m = e - q * N;
            float2& td = cTd[(g0 + q) * N + m];
            td = fftd::new_direction(fbuf[q * G::LDR + fftd::sidx<MC>(m)], td, beta, restart);
        }
        __syncthreads();
    }
    if (!dir_aside) {
        direction_rows(A.g, R, cd, cg, beta, restart, threadIdx.x, kLoopThreads);
        __syncthreads();
    }
    ls_rows_any<true>(A.reg, R, cf, cd, cRes, cD, cTd, 0.f, acc, reinterpret_cast<float*>(fbuf),
                      ls_planes_fit(A.reg, R.nown * N, G::FBUF));
}

// ------------------------------------------------------------ phases D, E

// Steps 2 and 3 of the line search, from the planes the row pass left in
// the FFT buffer when they fit.
template <int MC>
__device__ __forceinline__ void phase_ls(const Reg& reg, const Rows& R, const float2* cf, const float2* cd,
                                         float2* fbuf, float t, float (&acc)[2])
{
    ls_rows_any<false>(reg, R, cf, cd, nullptr, nullptr, nullptr, t, acc, reinterpret_cast<float*>(fbuf),
                       ls_planes_fit(reg, R.nown * R.N, Geo<MC>::FBUF));
}

// ------------------------------------------------------------------ kernel

template <int MC>
__global__ void __launch_bounds__(kLoopThreads, 1) k_cg_loop(LoopArgs A)
{
    static_assert(MC > 0, "the loop kernel needs a compile-time FFT size");
    using G = Geo<MC>;
    extern __shared__ float2 sm[];
    __shared__ LoopShared S;
    const int N = A.N, RB = A.RB;
    Rows R;
    R.N = N;
    R.R0 = blockIdx.x * RB;
    R.nown = min(RB, N - R.R0);
    R.hlo = R.R0 > 0 ? R.R0 - 1 : R.R0;
    R.hhi = min(R.R0 + R.nown, N - 1);
    float2* fbuf = sm;
    float2* stw = fbuf + G::FBUF;     // staged twiddles of exp(-2 pi i k / M)
    float2* cf = stw + G::TW;         // rows R0-1 .. R0+RB: f
    float2* cd = cf + (RB + 2) * N;   // the same rows: d
    float2* cRes = cd + (RB + 2) * N;  // own rows: T f - D, D, g, T d
    float2* cD = cRes + RB * N;
    float2* cg = cD + RB * N;
    float2* cTd = cg + RB * N;
    float2* pbuf = cTd + RB * N;  // deferred update partials (kUpdVals x even (grid + 1))
    pbuf += ((uintptr_t)pbuf & 15) ? 1 : 0;  // 16-byte copies
    // column groups: the wide ones when every block still gets one
    const bool wide_cols = G::CBPT2 > G::CBPT && MC / G::CPC2 >= (int)gridDim.x;
    const int cpc = G::FOURSTEP ? G::FS_COLS : wide_cols ? G::CPC2 : G::CPC;
    const int col_groups = MC / cpc;
    // rows: two FFT groups per batch (the split FFTs of M = 1024 have no groups)
    const bool rx2 = !G::FOURSTEP && RB >= 2 * G::RPC;
    constexpr int RX2 = G::FOURSTEP ? 1 : 2;
    const bool prof = blockIdx.x == 0;
    unsigned seq = 0;
    float t_f = 0.f;  // the current line-search step, the same in every thread
    if (threadIdx.x == 0) {
        S.ss = A.scal[S_SS];
        for (int i = 0; i < kProf; ++i) S.prof[i] = 0;
    }
    // block 0 keeps, per phase, its work time and its synchronisation time
    auto mark = [&](int i) {
        if (prof && threadIdx.x == 0) {
            const uint64_t now = gtimer();
            S.prof[i] += now - S.tmark;
            S.tmark = now;
        }
    };

    // ---- caches: twiddles, f of the cached rows, T f - D and D of the own rows
    {
        if constexpr (G::FOURSTEP) {
            // T16[k2][l] = w512^(l k2) = w1024^(2 l k2); WN[j][l] = w1024^(l + 32 j)
            for (int e = threadIdx.x; e < 512; e += kLoopThreads) {
                stw[e] = __ldg(A.tw + ((2 * (e & 31) * (e >> 5)) & (MC - 1)));
                stw[512 + e] = __ldg(A.tw + e);
            }
        } else {
            fftd::build_staged_twiddles<MC>(A.tw, stw);
        }
        const int nc = (R.hhi - R.hlo + 1) * N;
        const float2* src = A.f0 + (int64_t)R.hlo * N;
        float2* dst = cf + R.cache(R.hlo);
        for (int e = threadIdx.x; e < nc; e += kLoopThreads) dst[e] = __ldcg(src + e);
        const int64_t o = (int64_t)R.R0 * N;
        for (int e = threadIdx.x; e < R.nown * N; e += kLoopThreads) {
            cRes[e] = __ldcg(A.res + o + e);
            cD[e] = __ldg(A.D + o + e);
        }
    }
    __syncthreads();
    if (A.stall) {
        // a test's injected stall: wait for one arrival more than the grid
        // makes, so that the bounded wait runs out in every block
        if (threadIdx.x == 0)
            S.ok = grid_arrive_wait(A.counter, gridDim.x + 1, A.abort_word, A.err, A.wait_ns) ? 1 : 0;
        __syncthreads();
        if (!S.ok) return;
    }

    // ---- gradient at x0, J(x0); the first direction is -g (beta = 0)
    {
        float a[kUpdVals] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (rx2)
            phase_update<MC, true, RX2>(A, R, fbuf, stw, cf, cd, cRes, cD, cg, cTd, 0.f, A.iters > 0, a);
        else
            phase_update<MC, true, 1>(A, R, fbuf, stw, cf, cd, cRes, cD, cg, cTd, 0.f, A.iters > 0, a);
        if (!grid_reduce<kUpdVals>(a, A.parts, L_A, seq, S, A.counter, A.abort_word, A.err, A.wait_ns)) return;
        if (threadIdx.x == 0) {
            for (int v = 0; v < kUpdVals; ++v) S.red[v] = ff_to_double(S.redf[v]);
            double J, beta;
            cgd::update_finish(S.red, S.ss, 0.0, true, &J, &beta);
            S.gg = S.red[0];
            S.J = J;
            S.beta = 0.0;
            S.beta_f = 0.f;
            S.restart = 1;
            S.tmark = gtimer();
            if (blockIdx.x == 0) A.Jdev[0] = J;
        }
        __syncthreads();
    }

    for (int k = 0; k < A.iters; ++k) {
        // the sums of the previous update (k > 0) arrive while the columns run
        const bool deferred = k > 0;
        bool fetch = deferred;  // issued once the first column group is staged
        auto fetch_parts = [&] {
            if (fetch) deferred_parts_fetch<kUpdVals>(A.parts, L_A, pbuf);
            fetch = false;
        };
        if constexpr (!G::FOURSTEP) fetch_parts();
        // ---- B: columns
        for (int gi = blockIdx.x; gi < col_groups; gi += gridDim.x) {
            const int x0 = gi * cpc;
            if constexpr (G::FOURSTEP)
                cols_split(A.X, N, x0, A.ChatS, stw, stw + 512, fbuf, fetch_parts);
            else if (wide_cols)
                fftd::cols_group<MC, G::CBPT2, 1>(A.X, N, N, x0, cpc, cpc, A.fp, stw, A.Chat, fbuf, nullptr);
            else
                fftd::cols_group<MC, G::CBPT, 1>(A.X, N, N, x0, cpc, cpc, A.fp, stw, A.Chat, fbuf, nullptr);
            // the next group refills fbuf (after the last one, the
            // synchronisation below starts with a block barrier)
            if (gi + (int)gridDim.x < col_groups) __syncthreads();
        }
        mark(0);
        // the synchronisation; meanwhile warps 1..6 sum the previous update's
        // partials and warp 7 forms J and beta from them (the column pass does
        // not need beta: T d = -T g + beta T d_old is formed in the row pass)
        fetch_parts();  // a block without a column group
        if (deferred) deferred_parts_sum<kUpdVals>(pbuf, S);
        else __syncthreads();
        ++seq;
        if (threadIdx.x == 0) S.ok = grid_arrive_wait(A.counter, seq * gridDim.x, A.abort_word, A.err, A.wait_ns) ? 1 : 0;
        if (deferred && (threadIdx.x >> 5) >= 1 && (threadIdx.x >> 5) <= kUpdVals + 1) {
            asm volatile("bar.sync 1, %0;" ::"r"(32 * (kUpdVals + 1)) : "memory");
            if (threadIdx.x == 32 * (kUpdVals + 1)) finish_update(A, S, k);
        }
        __syncthreads();
        if (!S.ok) return;
        mark(1);
        const float beta = S.beta_f;
        const bool restart = S.restart != 0;
        // ---- C: rows, direction, first line-search sums
        {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            if (rx2)
                phase_rows<MC, RX2>(A, R, fbuf, stw, cf, cd, cRes, cD, cg, cTd, beta, restart, acc);
            else
                phase_rows<MC, 1>(A, R, fbuf, stw, cf, cd, cRes, cD, cg, cTd, beta, restart, acc);
            mark(2);
            if (!grid_reduce<4>(acc, A.parts, L_C, seq, S, A.counter, A.abort_word, A.err, A.wait_ns)) return;
            // every thread forms t1 from the totals (no broadcast, no barrier);
            // thread 0 keeps q1, q2 and t1 for the next steps
            const FF t1 = cgd::ls_next_ff(FF{0.f, 0.f}, S.redf[0], S.redf[3], S.redf[1], S.redf[2]);
            t_f = t1.hi + t1.lo;
            if (threadIdx.x == 0) {
                S.q1 = S.redf[0];
                S.q2 = S.redf[3];
                S.tb[0] = t1;
            }
            mark(3);
        }
        // ---- D, E: majorize-minimize steps at t1 and t2
#pragma unroll 1
        for (int j = 0; j < 2; ++j) {
            float acc[2] = {0.f, 0.f};
            phase_ls<MC>(A.reg, R, cf, cd, fbuf, t_f, acc);
            mark(4 + 2 * j);
            if (!grid_reduce<2>(acc, A.parts, j == 0 ? L_D : L_E, seq, S, A.counter, A.abort_word, A.err, A.wait_ns)) return;
            // t2 from t1 (tb[0] -> tb[1]), then t3 from t2 (tb[1] -> tb[0]),
            // in every thread; the step read and the step written never share
            // a slot
            const FF tn = cgd::ls_next_ff(S.tb[j], S.q1, S.q2, S.redf[0], S.redf[1]);
            t_f = tn.hi + tn.lo;
            if (threadIdx.x == 0) S.tb[1 - j] = tn;
            mark(5 + 2 * j);
        }
        // ---- A: step, gradient, row FFTs of g for the next iteration
        {
            float a[kUpdVals] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (rx2)
                phase_update<MC, false, RX2>(A, R, fbuf, stw, cf, cd, cRes, cD, cg, cTd, t_f, k + 1 < A.iters, a);
            else
                phase_update<MC, false, 1>(A, R, fbuf, stw, cf, cd, cRes, cD, cg, cTd, t_f, k + 1 < A.iters, a);
            mark(8);
            if (!grid_arrive_parts<kUpdVals>(a, A.parts, L_A, seq, S, A.counter, A.abort_word, A.err, A.wait_ns)) return;
            mark(9);
        }
    }
    // ---- J and beta of the last update
    if (A.iters > 0) {
        const int warp = threadIdx.x >> 5;
        if (warp < kUpdVals) {
            const FF a = warp_sum_parts(A.parts + (L_A + warp) * kMaxParts, gridDim.x);
            if ((threadIdx.x & 31) == 0) S.red[warp] = ff_to_double(a);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            finish_update(A, S, A.iters);
            if (blockIdx.x == 0) {  // the last iteration's line-search scalars
                A.scal[S_Q1] = ff_to_double(S.q1);
                A.scal[S_Q2] = ff_to_double(S.q2);
                A.scal[S_T3] = ff_to_double(S.tb[0]);
            }
        }
        __syncthreads();
    }
    // ---- the iterate and T f - D back to global memory
    {
        const int64_t o = (int64_t)R.R0 * N;
        const float2* fo = cf + R.cache(R.R0);
        for (int e = threadIdx.x; e < R.nown * N; e += kLoopThreads) {
            A.f0[o + e] = fo[e];
            A.res[o + e] = cRes[e];
        }
    }
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        for (int i = 0; i < kProf; ++i) A.scal[S_PROF + i] = (double)S.prof[i];
        A.scal[S_GG] = S.gg;
        A.scal[S_BETA] = S.beta;
        A.scal[S_J] = S.J;
    }
}

// Sets the function's shared-memory cap (once per device, to the largest
// size any shape may ask for) and returns it.
template <int MC>
bool loop_cap(size_t* cap_out)
{
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return false;
    auto kern = k_cg_loop<MC>;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return false;
    const size_t cap = (size_t)optin - fa.sharedSizeBytes;
    // the cap is a property of the function shared by every plan and thread:
    // set once to the largest shape, never lowered (a concurrent launch with
    // a larger shape would fail)
    static std::mutex mu;
    static int set_cap[64] = {0};
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return false;
    if (set_cap[dev] < (int)cap) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap) != cudaSuccess)
            return false;
        set_cap[dev] = (int)cap;
    }
    *cap_out = cap;
    return true;
}

// Whether blocks of RB rows fit: shared memory within the cap and every
// block of the grid co-resident (the grid synchronisations need that).
template <int MC>
bool loop_fits(int N, int RB, size_t cap, int sms, int* grid_out, size_t* smem_out)
{
    const int grid = (N + RB - 1) / RB;
    const size_t smem = loop_smem<MC>(N, RB);
    if (smem > cap) return false;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_loop<MC>, kLoopThreads, smem) != cudaSuccess)
        return false;
    if (per_sm < 1 || grid > sms * per_sm || grid > kMaxParts) return false;
    *grid_out = grid;
    *smem_out = smem;
    return true;
}

// The shapes RB = gpb * RPC, gpb = 1 .. kMaxGroupsPerBlock (up to the first
// that holds the whole image), that fit; at most max.
template <int MC>
int loop_shapes(int N, int* RB, int* grid, int max)
{
    int sms = 0;
    size_t cap = 0;
    if (device_sms(&sms) != SPIREC_OK || !loop_cap<MC>(&cap)) return 0;
    int n = 0;
    for (int gpb = 1; gpb <= kMaxGroupsPerBlock && n < max; ++gpb) {
        const int rb = gpb * Geo<MC>::RPC;
        int gr = 0;
        size_t smem = 0;
        if (loop_fits<MC>(N, rb, cap, sms, &gr, &smem)) {
            RB[n] = rb;
            grid[n] = gr;
            ++n;
        }
        if (rb >= N) break;
    }
    cudaGetLastError();
    return n;
}

// The block shape of a launch: the tuned rows per block of the plan's shape
// when that fits, else the fewest groups per block gpb whose grid is
// co-resident (every block on its own SM when the image allows).
template <int MC>
bool loop_shape(const spirec_plan_s* p, int* RB_out, int* grid_out, size_t* smem_out)
{
    int sms = 0;
    size_t cap = 0;
    if (device_sms(&sms) != SPIREC_OK || !loop_cap<MC>(&cap)) return false;
    const int N = p->N;
    const int tuned = tune_lookup(SPIREC_KNOB_LOOP_ROWS, p, sms);
    if (tuned > 0 && loop_fits<MC>(N, tuned, cap, sms, grid_out, smem_out)) {
        *RB_out = tuned;
        return true;
    }
    for (int gpb = 1; gpb <= kMaxGroupsPerBlock; ++gpb) {
        const int RB = gpb * Geo<MC>::RPC;
        if (loop_fits<MC>(N, RB, cap, sms, grid_out, smem_out)) {
            *RB_out = RB;
            return true;
        }
        if (RB >= N) return false;
    }
    return false;
}

// The spectrum in the split order of the M = 1024 column pass:
// out[c * 1024 + h * 512 + k] = Chat[kx * 1024 + 2 k + h], kx = 2 (c mod 512) + c / 512
// (column c of the split row layout holds the frequency kx).
__global__ void k_chat_split(const float* __restrict__ Chat, float* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // < 1024 * 1024
    const int c = i >> 10, h = (i >> 9) & 1, k = i & 511;
    const int kx = 2 * (c & 511) + (c >> 9);
    out[i] = __ldg(Chat + kx * 1024 + 2 * k + h);
}

struct LaunchLoop {
    spirec_plan p;
    int iters;
    template <int MC>
    int operator()()
    {
        if constexpr (MC == 0) {
            set_error("no compile-time FFT size for M=%d", p->M);
            return SPIREC_EUNSUPPORTED;
        } else {
            int RB = 0, grid = 0;
            size_t smem = 0;
            if (!loop_shape<MC>(p, &RB, &grid, &smem)) {
                cudaGetLastError();
                set_error("the persistent loop does not fit N=%d, M=%d", p->N, p->M);
                return SPIREC_EUNSUPPORTED;
            }
            LoopArgs A{};
            A.N = p->N;
            A.iters = iters;
            A.RB = RB;
            A.f0 = p->f[0];
            A.g = p->g;
            A.res = p->res;
            A.D = p->D;
            A.X = p->X;
            A.Chat = p->Chat;
            if constexpr (Geo<MC>::FOURSTEP) {
                // the split-order copy, in the spectrum build's scratch (M x M complex)
                float* chs = reinterpret_cast<float*>(p->cwork);
                k_chat_split<<<1024 * 1024 / 256, 256, 0, p->stream>>>(p->Chat, chs);
                SPIREC_CK(cudaGetLastError());
                p->launches += 1;
                A.ChatS = chs;
            }
            A.tw = p->twiddle;
            A.fp = p->fft;
            A.reg = p->reg;
            A.scal = p->scal;
            A.Jdev = p->Jdev;
            A.parts = reinterpret_cast<float2*>(p->part);
            A.counter = p->counters + C_BAR;
            A.abort_word = p->counters + C_BAR + 2;
            A.err = p->dflag;
            A.wait_ns = wait_limit_ns();
            A.stall = injected_stall(kStallLoop) ? 1 : 0;
            // no arrivals, no abort
            SPIREC_CK(cudaMemsetAsync(A.counter, 0, 3 * sizeof(unsigned), p->stream));
            void* args[] = {&A};
            SPIREC_CK(cudaLaunchCooperativeKernel((const void*)k_cg_loop<MC>, dim3(grid), dim3(kLoopThreads), args,
                                                  smem, p->stream));
            p->launches += 1;
            return SPIREC_OK;
        }
    }
};

}  // namespace

bool loop_supported(int M) { return M >= 64 && M <= 2048 && (M & (M - 1)) == 0; }

namespace {
struct Shapes {
    const spirec_plan_s* p;
    int* RB;
    int* grid;
    int max;
    bool current;
    int* capacity;  // with current: co-resident blocks the device holds of that shape
    template <int MC>
    int run()
    {
        if constexpr (MC == 0) {
            return 0;
        } else {
            if (current) {
                size_t smem = 0;
                if (!loop_shape<MC>(p, RB, grid, &smem)) return 0;
                if (capacity) {
                    int sms = 0, per_sm = 0;
                    if (device_sms(&sms) != SPIREC_OK ||
                        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_loop<MC>, kLoopThreads, smem) !=
                            cudaSuccess) {
                        cudaGetLastError();
                        return 0;
                    }
                    *capacity = sms * per_sm;
                }
                return 1;
            }
            return loop_shapes<MC>(p->N, RB, grid, max);
        }
    }
};

int shapes_for(const spirec_plan_s* p, int* RB, int* grid, int max, bool current, int* capacity = nullptr)
{
    Shapes s{p, RB, grid, max, current, capacity};
    switch (p->M) {
    case 64: return s.run<64>();
    case 128: return s.run<128>();
    case 256: return s.run<256>();
    case 512: return s.run<512>();
    case 1024: return s.run<1024>();
    case 2048: return s.run<2048>();
    default: return s.run<0>();
    }
}
}  // namespace

int loop_candidates(spirec_plan p, int* RB, int* grid, int max) { return shapes_for(p, RB, grid, max, false); }

int loop_current(spirec_plan p, int* RB, int* grid) { return shapes_for(p, RB, grid, 1, true); }

int loop_demand(spirec_plan p, int* blocks, int* capacity)
{
    int RB = 0;
    *blocks = 0;
    *capacity = 0;
    if (!loop_supported(p->M)) return 0;
    return shapes_for(p, &RB, blocks, 1, true, capacity);
}

int launch_cg_loop(spirec_plan p, int iters)
{
    switch (p->M) {
    case 64: return LaunchLoop{p, iters}.operator()<64>();
    case 128: return LaunchLoop{p, iters}.operator()<128>();
    case 256: return LaunchLoop{p, iters}.operator()<256>();
    case 512: return LaunchLoop{p, iters}.operator()<512>();
    case 1024: return LaunchLoop{p, iters}.operator()<1024>();
    case 2048: return LaunchLoop{p, iters}.operator()<2048>();
    default: return LaunchLoop{p, iters}.operator()<0>();
    }
}

}  // namespace spirec
