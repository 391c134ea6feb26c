// cg_loop.cu -- the whole Polak-Ribiere loop (section 3.3 on the rewritten
// criterion of section 3.4) as ONE persistent cooperative kernel.
//
// Two 512-thread blocks per SM, resident for the whole solve.  Each iteration
// runs the six phases of the stand-alone path (fft.cu, cg.cu), separated by
// grid barriers instead of kernel boundaries:
//   P1 rows:    d = -g + beta d_old, q1, line-search sums at t = 0, row FFTs
//   P2 columns: FFT * Chat * IFFT
//   P3 rows:    row IFFTs -> T d, q2            -> t1
//   P4, P5:     line-search steps at t1, t2     -> t2, t3
//   P6:         f += t3 d, T f += t3 T d, g, J  -> beta
// After each reducing phase every block sums the per-block partials itself
// (same order in every block), so all blocks hold the same FP64 scalars and
// no extra barrier is needed to broadcast them.  Partials of consecutive
// phases use different slots, so a fast block never overwrites a partial a
// slow block is still reading.
//
// The grid barrier is an arrival counter plus a generation word in global
// memory.  Its wait is bounded in time: on expiry the block raises an abort
// word and an error bit, every block returns at its next barrier, and the
// host reports SPIREC_ETIMEOUT.  The cooperative launch guarantees that all
// blocks are resident, so the barrier cannot wait on an unscheduled block.
#include <stdint.h>

#include "cg_device.cuh"
#include "fft_device.cuh"
#include "internal.cuh"
#include "reduce.cuh"

namespace spirec {

namespace {

constexpr int kLoopThreads = 512;
constexpr unsigned long long kBarrierNs = 2000000000ull;  // 2 s

struct LoopArgs {
    int N, iters;
    float2* f[2];
    float2* dbuf[2];
    float2* g;
    float2* Tf;
    float2* Td;
    const float2* D;
    float2* X;
    const float* Chat;
    const float2* tw;
    FftPlan fp;
    Reg reg;
    double* scal;
    double* Jdev;
    float2* parts;
    unsigned* bar;  // [0] arrivals, [1] generation, [2] abort
    int* err;
};

__device__ __forceinline__ uint64_t gtimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier; false (in every thread of the block) after an abort or
// a timeout.  Arrival is a release add, the wait an acquire load, so the
// block's writes (ordered before thread 0 by the __syncthreads) are visible
// to every block that passes, without separate full fences.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned& gen, int* err)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned g = gen;
        unsigned old;
        asm volatile("atom.add.release.gpu.u32 %0, [%1], 1;" : "=r"(old) : "l"(bar) : "memory");
        if (old == gridDim.x - 1) {
            asm volatile("st.relaxed.gpu.u32 [%0], 0;" ::"l"(bar) : "memory");
            asm volatile("st.release.gpu.u32 [%0], %1;" ::"l"(bar + 1), "r"(g + 1) : "memory");
        } else {
            const uint64_t t0 = gtimer();
            for (;;) {
                unsigned cur, ab;
                asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(cur) : "l"(bar + 1) : "memory");
                if (cur != g) break;
                asm volatile("ld.relaxed.gpu.u32 %0, [%1];" : "=r"(ab) : "l"(bar + 2) : "memory");
                if (ab) {
                    ok = 0;
                    break;
                }
                if (gtimer() - t0 > kBarrierNs) {
                    atomicExch(&bar[2], 1u);
                    atomicOr(err, E_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(20);
            }
        }
        gen = g + 1;
    }
    __syncthreads();
    return ok != 0;
}

// Block partials of K values to parts slot `slot`, barrier, then the grid
// totals (index order, float-float) in every thread as FP64.
template <int K>
__device__ __forceinline__ bool grid_reduce(float (&v)[K], float2* parts, int slot, unsigned* bar,
                                            unsigned& gen, int* err, double (&out)[K])
{
    __shared__ double bc[K];
    FF bt[K];
    block_partial<K>(v, bt);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; ++k)
            parts[(slot + k) * kMaxParts + blockIdx.x] = make_float2(bt[k].hi, bt[k].lo);
    if (!grid_barrier(bar, gen, err)) return false;
    // warp k sums value k over the blocks
    const int warp = threadIdx.x >> 5;
    if (warp < K) {
        const FF a = warp_sum_parts(parts + (slot + warp) * kMaxParts, gridDim.x);
        if ((threadIdx.x & 31) == 0) bc[warp] = ff_to_double(a);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = bc[k];
    __syncthreads();
    return true;
}

// partial slots of the loop (distinct per consecutive phase)
constexpr int L_P1 = 0;   // 3
constexpr int L_P3 = 3;   // 1
constexpr int L_P4 = 4;   // 2
constexpr int L_P5 = 6;   // 2
constexpr int L_P6 = 8;   // 6

template <int MC>
__global__ void __launch_bounds__(kLoopThreads, 2) k_cg_loop(LoopArgs A)
{
    static_assert(MC > 0, "the loop kernel needs a compile-time FFT size");
    extern __shared__ float2 sm[];
    constexpr int RPC = 4 * kLoopThreads / MC;  // rows per group: 512 threads = RPC * MC / 4
    constexpr int CBPT = MC >= 256 ? 2 : 1;      // column groups: CBPT butterflies per thread
    constexpr int CPC = CBPT * RPC;
    const int N = A.N, M = MC;
    const int P = N * N;
    const int row_groups = (N + RPC - 1) / RPC;
    const int col_groups = (M + CPC - 1) / CPC;
    const Reg reg = A.reg;
    unsigned gen = 0;
    if (threadIdx.x == 0) gen = *(volatile unsigned*)&A.bar[1];
    // block 0 keeps, per phase, its work time and its barrier+reduce time
    const bool prof = blockIdx.x == 0 && threadIdx.x == 0;
    uint64_t tprof[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    uint64_t tmark = prof ? gtimer() : 0;
    auto mark = [&](int i) {
        if (prof) {
            const uint64_t now = gtimer();
            tprof[i] += now - tmark;
            tmark = now;
        }
    };

    // ---- gradient at x0, J(x0); the first direction is -g (beta = 0)
    double ss = A.scal[S_SS];
    double gg, beta, J;
    {
        float a[kUpdVals];
#pragma unroll
        for (int i = 0; i < kUpdVals; ++i) a[i] = 0.f;
        for (int p = blockIdx.x * kLoopThreads + threadIdx.x; p < P; p += gridDim.x * kLoopThreads)
            cgd::update_pixel<true>(p, N, A.f[0], A.f[0], A.dbuf[1], A.Tf, A.Td, A.D, A.g, reg, 0.f, a);
        double s[kUpdVals];
        if (!grid_reduce<kUpdVals>(a, A.parts, L_P6, A.bar, gen, A.err, s)) return;
        cgd::update_finish(s, ss, 0.0, true, &J, &beta);
        gg = s[0];
        if (blockIdx.x == 0 && threadIdx.x == 0) A.Jdev[0] = J;
    }

    for (int k = 0; k < A.iters; ++k) {
        const float2* fin = A.f[k & 1];
        float2* fout = A.f[(k + 1) & 1];
        float2* dk = A.dbuf[k & 1];
        // ---- P1
        CgPass c{};
        c.g = A.g;
        c.d_old = A.dbuf[(k + 1) & 1];
        c.d_new = dk;
        c.f = fin;
        c.Tf = A.Tf;
        c.D = A.D;
        c.reg = reg;
        double q1, num0, den0;
        {
            float acc[3] = {0.f, 0.f, 0.f};
            for (int gi = blockIdx.x; gi < row_groups; gi += gridDim.x) {
                const int r0 = gi * RPC;
                fftd::rows_fwd_group<MC, 1>(nullptr, N, N, r0, min(RPC, N - r0), RPC, A.X, A.fp, A.tw, c,
                                            (float)beta, beta == 0.0, sm, nullptr, acc);
            }
            mark(0);
            double s[3];
            if (!grid_reduce<3>(acc, A.parts, L_P1, A.bar, gen, A.err, s)) return;
            q1 = s[0];
            num0 = s[1];
            den0 = s[2];
            mark(1);
        }
        // ---- P2
        for (int gi = blockIdx.x; gi < col_groups; gi += gridDim.x) {
            const int x0 = gi * CPC;
            fftd::cols_group<MC, CBPT>(A.X, N, N, x0, min(CPC, M - x0), CPC, A.fp, A.tw, A.Chat, sm, nullptr);
        }
        mark(2);
        if (!grid_barrier(A.bar, gen, A.err)) return;
        mark(3);
        // ---- P3
        double q2, t;
        {
            float acc[1] = {0.f};
            for (int gi = blockIdx.x; gi < row_groups; gi += gridDim.x) {
                const int r0 = gi * RPC;
                fftd::rows_inv_group<MC>(A.X, r0, min(RPC, N - r0), RPC, A.Td, N, A.fp, A.tw, dk, sm, nullptr,
                                         acc[0]);
            }
            mark(4);
            double s[1];
            if (!grid_reduce<1>(acc, A.parts, L_P3, A.bar, gen, A.err, s)) return;
            q2 = s[0];
            const double curv = 2.0 * q2 + den0;
            t = curv > 0.0 ? -(q1 + num0) / curv : 0.0;
            mark(5);
        }
        // ---- P4, P5: majorize-minimize steps at t1 and t2
#pragma unroll 1
        for (int j = 0; j < 2; ++j) {
            float acc[2] = {0.f, 0.f};
            const float tf = (float)t;
            for (int p = blockIdx.x * kLoopThreads + threadIdx.x; p < P; p += gridDim.x * kLoopThreads)
                cgd::ls_pixel(p, N, fin, dk, reg, tf, acc[0], acc[1]);
            mark(6 + 2 * j);
            double s[2];
            if (!grid_reduce<2>(acc, A.parts, j == 0 ? L_P4 : L_P5, A.bar, gen, A.err, s)) return;
            t = cgd::ls_next(t, q1, q2, s[0], s[1]);
            mark(7 + 2 * j);
        }
        // ---- P6
        {
            float a[kUpdVals];
#pragma unroll
            for (int i = 0; i < kUpdVals; ++i) a[i] = 0.f;
            const float tf = (float)t;
            for (int p = blockIdx.x * kLoopThreads + threadIdx.x; p < P; p += gridDim.x * kLoopThreads)
                cgd::update_pixel<false>(p, N, fin, fout, dk, A.Tf, A.Td, A.D, A.g, reg, tf, a);
            mark(10);
            double s[kUpdVals];
            if (!grid_reduce<kUpdVals>(a, A.parts, L_P6, A.bar, gen, A.err, s)) return;
            cgd::update_finish(s, ss, gg, false, &J, &beta);
            gg = s[0];
            mark(11);
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                A.Jdev[k + 1] = J;
                A.scal[S_Q1] = q1;
                A.scal[S_Q2] = q2;
                A.scal[S_T3] = t;
            }
        }
    }
    if (prof)
        for (int i = 0; i < 12; ++i) A.scal[S_PROF + i] = (double)tprof[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.scal[S_GG] = gg;
        A.scal[S_BETA] = beta;
        A.scal[S_J] = J;
    }
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
            constexpr int RPC = 4 * kLoopThreads / MC;
            constexpr int CPC = (MC >= 256 ? 2 : 1) * RPC;
            const size_t smem = (size_t)CPC * (fftd::seq_len<MC>(MC) + 4) * sizeof(float2);
            auto kern = k_cg_loop<MC>;
            SPIREC_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            int dev = 0, sms = 0, per_sm = 0;
            SPIREC_CK(cudaGetDevice(&dev));
            SPIREC_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            SPIREC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLoopThreads, smem));
            if (per_sm < 1) {
                set_error("loop kernel does not fit on an SM");
                return SPIREC_EUNSUPPORTED;
            }
            // about two pixels per thread: the whole GPU at 512^2, a fraction of
            // it for small images, so loops of concurrent solves can co-reside
            int grid = (int)(((int64_t)p->N * p->N + 2 * kLoopThreads - 1) / (2 * kLoopThreads));
            if (grid > sms * per_sm) grid = sms * per_sm;
            if (grid > kMaxParts) grid = kMaxParts;
            if (grid < 1) grid = 1;
            LoopArgs A{};
            A.N = p->N;
            A.iters = iters;
            A.f[0] = p->f[0];
            A.f[1] = p->f[1];
            A.dbuf[0] = p->dbuf[0];
            A.dbuf[1] = p->dbuf[1];
            A.g = p->g;
            A.Tf = p->Tf;
            A.Td = p->Td;
            A.D = p->D;
            A.X = p->X;
            A.Chat = p->Chat;
            A.tw = p->twiddle;
            A.fp = p->fft;
            A.reg = p->reg;
            A.scal = p->scal;
            A.Jdev = p->Jdev;
            A.parts = reinterpret_cast<float2*>(p->part);
            A.bar = p->counters + C_BAR;
            A.err = p->dflag;
            // arrivals and abort start at zero; the generation word carries over
            SPIREC_CK(cudaMemsetAsync(A.bar, 0, sizeof(unsigned), p->stream));
            SPIREC_CK(cudaMemsetAsync(A.bar + 2, 0, sizeof(unsigned), p->stream));
            void* args[] = {&A};
            SPIREC_CK(cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(kLoopThreads), args, smem,
                                                  p->stream));
            p->launches += 1;
            return SPIREC_OK;
        }
    }
};

}  // namespace

bool loop_supported(int M) { return M >= 64 && M <= 2048 && (M & (M - 1)) == 0; }

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
