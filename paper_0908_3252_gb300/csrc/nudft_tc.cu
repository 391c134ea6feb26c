// nudft_tc.cu -- tensor-core (tcgen05, sm_103a) contractions of the exact
// NUDFT: G (Eq. AnnMatG), D = H^H s (Eq. AnnMatGD) and the forward H f
// (Eq. ModDirect).
//
// G and D are complex GEMMs C[i][c] = sum_l A(l,i) B(l,c) of depth K = L
// whose operands are phases generated on the fly (phase.cuh).  The B
// operand's phases come in conjugate pairs: exp(-i x) = conj(exp(i x)), so
// output columns mirrored about a centre share one set of four real
// products (PairGeom)
//      P_ac = Ar Br^T   P_bd = Ai Bi^T   P_ad = Ar Bi^T   P_bc = Ai Br^T
// and the drain forms both columns, (P_ac - P_bd, P_ad + P_bc) and (P_ac +
// P_bd, P_bc - P_ad).  G needs its lags v and -v, D its columns on both sides
// of the image centre: half the MMAs of forming every column on its own.
// The kernel runs on CTA pairs (clusters of two, one CTA per SM).  A pair
// tile is 256 rows x 128 B columns; CTA h holds A rows 128 h .. 128 h + 127
// (real and imaginary parts as two operand tiles) and, for B columns 64 h ..
// 64 h + 63, B stored once as a stacked operand of 128 rows [Br ; Bi].  Two
// pair MMAs (tcgen05.mma.cta_group::2, M = 256, N = 256) per K slice, A_re
// [B]^T = [P_ac | P_ad] and A_im [B]^T = [P_bc | P_bd] per B half, read both
// CTAs' tiles and fill all 512 columns of each CTA's tensor memory for its
// 128 rows.  N = 256 reads 12 KB of shared memory per 128 x 256 x 16 product
// where two N = 128 MMAs read 16 KB (the tensor core's operand reads and the
// producers' stores share the shared-memory data path), and the pair halves
// the B columns each SM generates.
//
// Split precision: every operand value x is stored as x_hi = fp16(x) (or
// bf16) and x_lo = fp16(x - x_hi); the products hi*hi + hi*lo + lo*hi feed
// the same FP32 accumulator (the dropped lo*lo term is 2^-22 relative for
// FP16).
//
// Work split (stream-K): the pair tiles x sample-chunks units are cut into
// equal contiguous ranges, one per pair and one pair per two SMs, so every
// SM does the same work whatever the tile count; a range may end in one tile
// and go on in the next.  CTA h of pair c writes its rows' partial of tile t
// to slot 2 (c + t) + h (unique, since c and t grow along the ranges) and
// k_reduce_pair adds the partials of each tile in pair order.
//
// Pipeline per CTA (544 threads):
//   warps 0-15 producers: per stage of 32 samples, each thread of warps 0-7
//              forms the phasors of two A rows (times the weight, for D) and
//              each thread of warps 8-15 those of one B column, for 8
//              samples (exact fixed-point phase, fast hardware sin/cos), so
//              a warp's 32 lanes share the 8 trajectory values they read;
//              splits them into hi and lo operand tiles in the
//              64-byte-swizzled K-major layout the MMA reads (rows of 32
//              samples), then each warp arrives once on the pair leader's
//              full[stage];
//   warp 16    allocates 512 TMEM columns (with the other CTA's warp 16); in
//              the leader, one lane waits on full[stage], issues 12 pair
//              MMAs (K = 16 each) and commits to empty[stage] of both CTAs;
//   warps 0-15 drain: at the end of every segment (at most SEG stages of one
//              tile) the finished accumulators are read with tcgen05.ld and
//              the paired outputs added to the CTA's partial tile in global
//              memory by fire-and-forget vector reductions
//              (red.global.add.v4.f32, round-to-nearest; the first segment
//              of a tile stores), laid out so that a warp's 32 lanes cover
//              512 contiguous bytes.  The leader's MMA waits for the drains
//              of both CTAs.
// The tensor core's FP32 accumulation loses about one unit in the last place
// per accumulation step (truncation-like, measured: 2.8e-4 relative after
// 12k steps); draining every 32 stages (384 accumulation steps) bounds that
// error.  Four stages of 48 KB buffer generation against the tensor core.
// The stage's 32 samples of the trajectory (and of the weights, for D) arrive
// by TMA bulk copy (cp.async.bulk) into an 8-deep shared-memory ring two
// stages ahead, so the table builders never wait on global memory.
// Every mbarrier wait is bounded in time; on expiry the kernel records an
// error bit, lets the other roles run out, waits for its own copies and
// MMAs, meets the other CTA of its pair, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "internal.cuh"
#include "phase.cuh"

namespace spirec {

namespace {

constexpr int TC_ROWS = 128;        // complex rows per tile (MMA M)
constexpr int TC_COLS = 256;        // complex columns per tile (MMA N)
constexpr int TC_KS = 32;           // samples per stage
constexpr int TC_STAGES = 2;
constexpr int TC_PRODUCERS = 512;   // 16 warps
constexpr int TC_THREADS = TC_PRODUCERS + 32;
constexpr int TC_SEG = 32;          // stages per accumulator segment (at most)
constexpr int TC_TILE_FLOATS = 2 * TC_COLS * TC_ROWS;  // partial tile: 512 columns x 128 rows
constexpr uint32_t A_BYTES = TC_ROWS * 128;          // 128 rows x 64 halves
constexpr uint32_t B_BYTES = TC_COLS * 128;          // 256 rows x 64 halves
constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;  // A_hi, A_lo, B_hi, B_lo
// The paired contraction (G, D): a tile is ROWS rows x 128 B columns, each B
// column giving two output columns (see PairGeom).  The operands are stored
// in 64-byte-swizzled K-major tiles of 32 samples per row: A's real and
// imaginary parts as two tiles of 128 rows, B as a stacked tile [Br ; Bi] of
// the BCOLS columns a CTA generates.  Two tile shapes (the tile knob):
//   one SM a tile (PAIR = false): 128 rows; the CTA generates all 128 B
//     columns (256 stacked rows); MMA M = 128, N = 256 (cta_group::1);
//     three 64 KB stages;
//   a CTA pair a tile (PAIR = true, clusters of two): 256 rows, CTA h holding
//     rows 128 h .. +127 and B columns 64 h .. +63 (128 stacked rows); MMA
//     M = 256, N = 256 (cta_group::2) issued by the pair's first CTA; four
//     48 KB stages.
// Either way each CTA's TMEM holds its 128 rows of [P_ac | P_ad] and
// [P_bc | P_bd] (512 columns); the trajectory (and weight) chunks arrive in
// an 8-deep ring, two stages ahead.
constexpr int PG_COLS = 128;                                       // B columns per tile
constexpr uint32_t PA_BYTES = TC_ROWS * 64;                        // 128 rows x 32 halves
constexpr int PG_TRAJ_RING = 8;  // >= stages + 2: a slot is refilled only after every producer left it
constexpr uint32_t PG_TRAJ_BUF = 3 * TC_KS * 8;  // ka, kb (int64), w' (float2)
template <bool PAIR>
struct PairShape {
    static constexpr int ROWS = PAIR ? 2 * TC_ROWS : TC_ROWS;        // output rows per tile
    static constexpr int BCOLS = PAIR ? PG_COLS / 2 : PG_COLS;       // B columns a CTA generates
    static constexpr uint32_t B_TILE = 2 * BCOLS * 64;                // stacked rows x 32 halves
    static constexpr uint32_t STAGE = 4 * PA_BYTES + 2 * B_TILE;      // Ar, Ai (hi, lo), B (hi, lo)
    static constexpr int STAGES = PAIR ? 4 : 3;
    static constexpr uint32_t TRAJ_OFF = STAGES * STAGE;
    static constexpr uint32_t BAR_OFF = TRAJ_OFF + PG_TRAJ_RING * PG_TRAJ_BUF;
    static constexpr uint32_t SMEM = BAR_OFF + 256 + 1024;            // + 1024 alignment slack
    static constexpr int ARRIVALS = (PAIR ? 2 : 1) * TC_PRODUCERS / 32;  // producer warps feeding one MMA issuer
    static_assert(SMEM <= 232448, "shared memory per CTA");
    static_assert(PG_TRAJ_RING >= STAGES + 2, "trajectory ring depth");
    static_assert(8 * (2 * STAGES + 3 + PG_TRAJ_RING) + 8 <= 256, "barrier area");
};
constexpr int kMaxCtas = 152;       // CTAs of one contraction (one per SM)

// Every pipeline wait is bounded by the launch's wait limit (a kernel
// argument, 2 s unless a test sets it); on expiry the CTA raises E_TIMEOUT and
// winds down.  Before it releases its TMEM and exits it waits, with this
// fixed bound, for the asynchronous work it issued (TMA copies into its shared
// memory, MMAs reading it and writing TMEM), so that nothing of it is in
// flight once the CTA is gone.
constexpr unsigned long long kDrainNs = 2000000000ull;
constexpr int kErrTimeout = E_TIMEOUT;

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false after limit_ns without the phase completing.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns)
{
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try(bar, parity)) return true;
        if (globaltimer() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// 1-D TMA bulk copy global -> shared, completion counted on `bar`.
// dst and src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void producers_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(TC_PRODUCERS) : "memory");
}

// producers_sync that also returns, to every producer alike, whether any of
// them passed v = true (a barrier with an OR reduction): a decision every
// producer takes the same way, as it must be before a named barrier.
__device__ __forceinline__ bool producers_any(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(TC_PRODUCERS)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), leading offset unused for this layout, version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | (64ull << 32) | (1ull << 46) |
           (2ull << 61);
}

// The same for a 64-byte swizzle (rows of 64 bytes, 8-row groups 512 bytes
// apart; layout type 4).
__device__ __forceinline__ uint64_t sdesc64(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | (32ull << 32) | (1ull << 46) |
           (4ull << 61);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bar)
                 : "memory");
}

// ------------------------------------------------ CTA-pair (cluster) helpers

// Arrives on the mbarrier at shared offset `bar` of CTA `rank` of the
// cluster, with the arrive's default semantics (release at CTA scope).  What
// the arrival publishes is shared memory for the pair's MMAs, made visible to
// the tensor core's proxy by the arriving warp's fence.proxy.async, and TMEM
// read by tcgen05.ld that has completed: no cluster-scope fence (which would
// also wait for the warp's outstanding global reductions) is needed.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar, uint32_t rank)
{
    asm volatile(
        "{\n\t.reg .b32 ra;\n\t"
        "mapa.shared::cluster.u32 ra, %0, %1;\n\t"
        "mbarrier.arrive.shared::cluster.b64 _, [ra];\n\t}" ::"r"(bar),
        "r"(rank)
        : "memory");
}

// Every thread of both CTAs of the pair (release / acquire at cluster scope;
// the non-aligned form: a warp need not be converged).
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// TMEM of a CTA pair: one warp of each CTA allocates (and frees) together.
__device__ __forceinline__ void tmem_alloc2(uint32_t slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc2(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// One MMA across the pair: A rows 0-127 and B rows 0 .. N/2 - 1 from this
// CTA's shared memory, A rows 128-255 and B rows N/2 .. N - 1 from the same
// offsets in the peer's; each CTA's TMEM receives its 128 rows.
__device__ __forceinline__ void mma2_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrives on the mbarrier at shared offset `bar` of both CTAs of the pair once
// the pair MMAs this thread issued have completed.
__device__ __forceinline__ void mma2_commit_pair(uint32_t bar)
{
    asm volatile(
        "{\n\t.reg .b16 m;\n\t"
        "mov.b16 m, 3;\n\t"
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], m;\n\t}" ::"r"(
            bar)
        : "memory");
}

// Four loads of 8 TMEM columns (t0.., t1.., t2.., t3.., the warp's 32 lanes)
// behind one wait: one round trip to tensor memory instead of four.
__device__ __forceinline__ void tmem_ld8x4(uint32_t t0, uint32_t t1, uint32_t t2, uint32_t t3, float* a, float* b,
                                           float* c, float* d)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%33];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%34];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24,%25,%26,%27,%28,%29,%30,%31}, [%35];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(t0), "r"(t1), "r"(t2), "r"(t3));
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        a[i] = __uint_as_float(r[i]);
        b[i] = __uint_as_float(r[8 + i]);
        c[i] = __uint_as_float(r[16 + i]);
        d[i] = __uint_as_float(r[24 + i]);
    }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    // load and wait in one statement: the registers are valid only after the wait
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint4 v)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w)
                 : "memory");
}

// Byte offset of 16-byte chunk `chunk` (0..7) of K-major row `row` in a
// 128-byte-swizzled tile whose base is 1024-aligned.
__device__ __forceinline__ uint32_t sw128(int row, int chunk)
{
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4));
}

// Byte offset of 16-byte chunk `chunk` (0..3) of K-major row `row` in a
// 64-byte-swizzled tile whose base is 1024-aligned: address bits 4-5 are
// XORed with bits 7-8.
__device__ __forceinline__ uint32_t sw64(int row, int chunk)
{
    return (uint32_t)((row >> 3) * 512 + (row & 7) * 64 + ((chunk ^ ((row >> 1) & 3)) << 4));
}

// hi/lo split of a pair: hi = the pair rounded to FP16 (BF16), packed (a in
// the low half); lo = (x - hi) rounded the same way, where x - hi is formed
// exactly in FP32 by one mixed-precision FMA per value (hi * -1 + x).
template <bool BF16>
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo)
{
    float la, lb;
    if (BF16) {
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(b), "f"(a));
        asm("{\n\t.reg .b16 h0, h1, m;\n\t"
            "mov.b32 {h0, h1}, %2;\n\t"
            "mov.b16 m, 0xBF80;\n\t"  // -1
            "fma.rn.f32.bf16 %0, h0, m, %3;\n\t"
            "fma.rn.f32.bf16 %1, h1, m, %4;\n\t}"
            : "=f"(la), "=f"(lb)
            : "r"(hi), "f"(a), "f"(b));
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(lb), "f"(la));
    } else {
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(b), "f"(a));
        asm("{\n\t.reg .f16 h0, h1, m;\n\t"
            "mov.b32 {h0, h1}, %2;\n\t"
            "mov.b16 m, 0xBC00;\n\t"  // -1
            "fma.rn.f32.f16 %0, h0, m, %3;\n\t"
            "fma.rn.f32.f16 %1, h1, m, %4;\n\t}"
            : "=f"(la), "=f"(lb)
            : "r"(hi), "f"(a), "f"(b));
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(lb), "f"(la));
    }
}

// hi/lo split of 8 values into 4 packed words each.
template <bool BF16>
__device__ __forceinline__ void split8(const float* x, uint4& hi, uint4& lo)
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) split2<BF16>(x[2 * q], x[2 * q + 1], h[q], l[q]);
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// exp(+i 2 pi k j) from the fixed-point k: kq * j mod 2^64 is the exact
// phase (two's complement wraps it), its top 32 bits a signed fraction of a
// cycle, and the fast hardware sin/cos runs on an argument in [-pi, pi)
// (absolute error about 4e-7, below the split-precision contraction's own).
__device__ __forceinline__ float2 phasor_fast(int64_t kq, int j)
{
    const uint64_t th = (uint64_t)kq * (uint64_t)(int64_t)j;
    const float ang = (float)(int)(th >> 32) * 1.4629180792671596e-09f;  // 2 pi / 2^32
    float sn, cs;
    __sincosf(ang, &sn, &cs);
    return make_float2(cs, sn);
}

// exp(+i 2 pi k s a) for the fixed-point k = hi 2^32 + lo, a count a >= 0
// and a sign s = +-1 folded into scale = s * 2 pi / 2^32: the top 32 bits of
// kq * a mod 2^64 are hi a + umulhi(lo, a) mod 2^32 (two integer
// multiply-adds), the signed fraction of a cycle; negating the angle
// conjugates the phasor.  `c` adds a constant to that fraction (a half-integer
// offset's kq / 2, see the B operand of k_tc_pair_gemm).  The same phase as
// phasor_fast up to one unit of the 32-bit fraction.
__device__ __forceinline__ float2 phasor_top(uint32_t lo, uint32_t hi, uint32_t c, uint32_t a, float scale)
{
    const uint32_t top = __umulhi(lo, a) + c + hi * a;
    float sn, cs;
    __sincosf((float)(int)top * scale, &sn, &cs);
    return make_float2(cs, sn);
}

__device__ __forceinline__ void st_global_v4(float* p, const float* v)
{
    asm volatile("st.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3])
                 : "memory");
}

// p[0..3] += v[0..3] at the memory (round-to-nearest FP32 adds, no reply).
__device__ __forceinline__ void red_global_v4(float* p, const float* v)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]),
                 "f"(v[3])
                 : "memory");
}

// 2^-e with 2^e >= sqrt(amax2): scales the weights into (-1, 1).
__device__ __forceinline__ float weight_scale_inv(const unsigned* amax2_bits)
{
    if (!amax2_bits) return 1.f;
    const float a = sqrtf(__uint_as_float(*amax2_bits));
    if (!(a > 0.f)) return 1.f;
    int e;
    frexpf(a, &e);
    return ldexpf(1.f, -e);
}

// Pairing of the output columns.  The B operand is a pure phase,
// E(l, j) = exp(sb i2pi kb_l (j + half/2)), and its conjugate is the phase of
// the mirrored column, so one set of four real products
//      P_ac = Ar Br^T   P_bd = Ai Bi^T   P_ad = Ar Bi^T   P_bc = Ai Br^T
// (A' = Ar + i Ai, E = Br + i Bi, summed over the samples) gives two output
// columns:
//      sum A' E       = (P_ac - P_bd) + i (P_ad + P_bc)   at column c+(j)
//      sum A' conj(E) = (P_ac + P_bd) + i (P_bc - P_ad)   at column c-(j)
// with c+-(j) = (C2 +- (2j + half)) / 2.  The weight of the original B operand
// and the phase of the centre column move into A (A' = w' A,
// w'_l = w_l exp(sb i2pi kb_l (C2 / 2 + ob)), k_pair_weights).
//   G (Eq. AnnMatG): columns v + N - 1, centre v = 0 (C2 = 2N - 2, half 0),
//     j = 0 .. N - 1: the lags v and -v, unweighted.
//   D (Eq. AnnMatGD): columns m, centre (N - 1) / 2 (C2 = N - 1); for even N
//     the offsets are half-integers (half 1, j = 0 .. N/2 - 1: m = N/2 + j
//     and N/2 - 1 - j), for odd N integers (half 0, j = 0 .. (N - 1)/2).
// A half-integer phase k (j + 1/2) is k j + k/2: the fixed-point k times j
// plus k shifted right by one bit (an error of 2^-65 cycles, and one unit of
// 2^-32 cycle from adding the two top words without the low words' carry).
struct PairGeom {
    int R, C;   // output rows and columns
    int C2;     // twice the centre column
    int half;   // offsets j + 1/2
    int J;      // B columns j = 0 .. J - 1
};

// Adds (first: stores) this CTA's 128 rows of the four products as the two
// paired outputs into its partial tile.  B column j (0..127) of the tile is
// row j % BCOLS (Br) and BCOLS + j % BCOLS (Bi) of the stacked operand of
// the tile's (j / BCOLS)-th CTA (the only one, or one of a pair), so with
// cb = 2 BCOLS (j / BCOLS) + j % BCOLS the accumulators hold P_ac at TMEM
// column cb, P_ad at cb + BCOLS, P_bc at 256 + cb and P_bd at 256 + BCOLS +
// cb.  The partial
// tile is laid out as [column / 4][row][column % 4] (256 complex columns:
// c+(j) at j, c-(j) at 128 + j; real parts in the first 256 float columns,
// imaginary in the next 256; 128 rows): a thread's four consecutive columns
// are one 16-byte vector, and a warp's 32 lanes (consecutive rows) cover 512
// contiguous bytes.  Fire-and-forget vector reductions; a thread's adds to
// one address come in program order, so the partial is the same sum on every
// run.
template <int BCOLS>
__device__ __forceinline__ void drain_pairs(uint32_t tacc, float* ptile, int warp, int lane, bool first)
{
    const int lbase = 32 * (warp & 3);
    const int quarter = warp >> 2;  // columns j = 32 quarter .. + 31
    const int row = lbase + lane;
#pragma unroll 1
    for (int cc = 0; cc < 32; cc += 8) {
        float ac[8], bd[8], ad[8], bc[8];
        const int j = 32 * quarter + cc;
        const uint32_t cb = 2u * BCOLS * (uint32_t)(j / BCOLS) + (uint32_t)(j % BCOLS);
        const uint32_t ta = tacc + ((uint32_t)lbase << 16) + cb;
        tmem_ld8x4(ta, ta + BCOLS, ta + 256, ta + 256 + BCOLS, ac, ad, bc, bd);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float pre[4], pim[4], mre[4], mim[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int x = 4 * h + e;
                pre[e] = ac[x] - bd[x];
                pim[e] = ad[x] + bc[x];
                mre[e] = ac[x] + bd[x];
                mim[e] = bc[x] - ad[x];
            }
            const int cg = (32 * quarter + cc) / 4 + h;  // column group of c+; c- is 32 groups further
            float* p_re = ptile + ((size_t)cg * TC_ROWS + row) * 4;
            float* p_im = ptile + ((size_t)(TC_COLS / 4 + cg) * TC_ROWS + row) * 4;
            float* m_re = ptile + ((size_t)(PG_COLS / 4 + cg) * TC_ROWS + row) * 4;
            float* m_im = ptile + ((size_t)(TC_COLS / 4 + PG_COLS / 4 + cg) * TC_ROWS + row) * 4;
            if (first) {
                st_global_v4(p_re, pre);
                st_global_v4(p_im, pim);
                st_global_v4(m_re, mre);
                st_global_v4(m_im, mim);
            } else {
                red_global_v4(p_re, pre);
                red_global_v4(p_im, pim);
                red_global_v4(m_re, mre);
                red_global_v4(m_im, mim);
            }
        }
    }
}

// B column j = j0 + c of the columns a CTA generates, for the samples 8g ..
// 8g + 7 (fixed-point k = khi 2^32 + klo, phase constant kc): Br into row c
// and Bi into row BCOLS + c of the stacked hi and lo tiles.  MASK zeroes
// samples from nvalid on and columns from J on.
template <bool BF16, bool MASK, int BCOLS>
__device__ __forceinline__ void pair_b_col(const uint32_t* klo, const uint32_t* khi, const uint32_t* kc, int j0,
                                           int c, int g, int J, int nvalid, float scb, uint32_t bH, uint32_t bL)
{
    float re[8], im[8];
    uint4 rh, rl, ih, il;
    const int jb = j0 + c;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        float2 z = phasor_top(klo[e], khi[e], kc[e], (uint32_t)jb, scb);
        if (MASK && (8 * g + e >= nvalid || jb >= J)) z = make_float2(0.f, 0.f);
        re[e] = z.x;
        im[e] = z.y;
    }
    split8<BF16>(re, rh, rl);
    split8<BF16>(im, ih, il);
    st_shared_v4(bH + sw64(c, g), rh);
    st_shared_v4(bL + sw64(c, g), rl);
    st_shared_v4(bH + sw64(BCOLS + c, g), ih);
    st_shared_v4(bL + sw64(BCOLS + c, g), il);
}

// The unit range [u0, u1) of CTA c among P over U units (tiles x chunks).
__host__ __device__ __forceinline__ int64_t unit_start(int64_t c, int64_t U, int64_t P) { return c * U / P; }

// Segment bookkeeping along a CTA's stages: a segment is at most TC_SEG
// stages of one tile.  Producers and the MMA issuer step it identically.
struct SegWalk {
    int K;
    int tile, kc;  // tile and chunk of the current stage's unit (units < 2^31)
    int seg = -1, pos = 0;
    bool first_of_tile = false;
    // the first unit u0 (one division; every later stage steps the chunk)
    __device__ __forceinline__ SegWalk(int64_t u0, int64_t K_)
        : K((int)K_), tile((int)(u0 / K_)), kc((int)(u0 % K_))
    {
    }
    // advance to stage it (called for it = 0, 1, 2, ...)
    __device__ __forceinline__ void step(int it)
    {
        bool new_tile = it == 0;
        if (it > 0 && ++kc == K) {
            kc = 0;
            ++tile;
            new_tile = true;
        }
        if (new_tile || pos == TC_SEG - 1) {
            first_of_tile = new_tile;
            ++seg;
            pos = 0;
        } else {
            ++pos;
        }
    }
    // stage it (current) closes its segment
    __device__ __forceinline__ bool closes(int it, int n) const
    {
        return it == n - 1 || kc == K - 1 || pos == TC_SEG - 1;
    }
};

// Partials of the tile owner c over its units [u0, u1) (unit = tile * K +
// chunk of 32 samples; tile = row tile of ROWS * tilesC + column tile of 128
// j):
//   A'(l,i) = w'_l exp(sa i2pi ka_l (i + oa)) (w' = 1 unweighted),
//   E(l,j)  = exp(sb i2pi kb_l (j + half/2)),
// the four real products of each into the two accumulators of each CTA.
// One SM a tile: owner c = CTA blockIdx.x, partial of tile t in slot c + t.
// CTA pairs: owner c = pair blockIdx.x / 2; CTA h = blockIdx.x % 2 (its rank
// in the cluster) forms A rows 128 h .. +127 and B columns 64 h .. +63 of
// each tile and keeps its rows' partial of tile t in slot 2 (c + t) + h.
// Rank 0 issues the pair's MMAs: it waits on its own full[stage] barrier, on
// which the producer warps of both CTAs arrive, and its commits arrive on the
// barrier at the same offset in both CTAs.
template <bool BF16, bool WEIGHTED, bool PAIR>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_tc_pair_gemm(const int64_t* __restrict__ ka, const int64_t* __restrict__ kb, const float2* __restrict__ w,
               const unsigned* __restrict__ amax2, int64_t L, int tilesC, int oa, int sa, int sb, int half, int J,
               int64_t K, int64_t U, float* __restrict__ part, int* err, unsigned long long wait_ns, int stall)
{
    using SH = PairShape<PAIR>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar_full = sbase + SH::BAR_OFF;            // stage filled (the MMA issuer's CTA)
    const uint32_t bar_empty = bar_full + 8 * SH::STAGES;     // stage consumed
    const uint32_t bar_acc_full = bar_empty + 8 * SH::STAGES; // segment accumulated
    const uint32_t bar_acc_empty = bar_acc_full + 8;          // accumulator drained (rank 0)
    const uint32_t bar_traj = bar_acc_empty + 8;              // PG_TRAJ_RING: trajectory chunk landed
    const uint32_t bar_drain = bar_traj + 8 * PG_TRAJ_RING;   // every MMA issued has completed
    const uint32_t misc = SH::BAR_OFF + 8 * (2 * SH::STAGES + 3 + PG_TRAJ_RING);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + misc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + misc + 4);
    const uint32_t traj_s = sbase + SH::TRAJ_OFF;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    // the launch's clusters are pairs of consecutive blocks
    const uint32_t rank = PAIR ? (blockIdx.x & 1u) : 0u;
    const int64_t pair = PAIR ? blockIdx.x >> 1 : blockIdx.x, P2 = PAIR ? gridDim.x >> 1 : gridDim.x;
    const int64_t u0 = unit_start(pair, U, P2);
    const int n = (int)(unit_start(pair + 1, U, P2) - u0);

    if (tid == 0) {
        for (int i = 0; i < SH::STAGES; ++i) {
            mbar_init(bar_full + 8 * i, SH::ARRIVALS);  // one arrival per producer warp (of the pair)
            mbar_init(bar_empty + 8 * i, 1);
        }
        mbar_init(bar_acc_full, 1);
        mbar_init(bar_acc_empty, SH::ARRIVALS);
        for (int r = 0; r < PG_TRAJ_RING; ++r) mbar_init(bar_traj + 8 * r, 1);
        mbar_init(bar_drain, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == TC_PRODUCERS / 32) {
        if constexpr (PAIR) tmem_alloc2(smem_u32(tmem_slot), 512);
        else tmem_alloc(smem_u32(tmem_slot), 512);
    }
    tc_fence_before();
    __syncthreads();
    if constexpr (PAIR) cluster_sync();  // both CTAs' barriers are initialised before any arrival from the other
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < TC_PRODUCERS / 32) {
        // ------------------------------------------------ producers
        const float wmul = WEIGHTED ? weight_scale_inv(amax2) : 1.f;
        // TMA feed of the trajectory (and weight) chunk of stage `it` into
        // its ring slot; stages are issued in order, kci is the chunk of the next
        int64_t kci = u0 % K;
        int issued = 0;  // stages whose chunk thread 0 has requested
        auto issue_traj = [&](int it) {
            ++issued;
            const int64_t l0 = kci * TC_KS;
            if (++kci == K) kci = 0;
            // the whole chunk, also past L: the plan's sample arrays have 32
            // entries of padding, the weights' padding is zero
            const uint32_t bytes = (uint32_t)TC_KS * 8;
            const uint32_t buf = traj_s + (uint32_t)(it % PG_TRAJ_RING) * PG_TRAJ_BUF;
            const uint32_t bar = bar_traj + 8 * (it % PG_TRAJ_RING);
            fence_proxy_async();
            mbar_expect_tx(bar, (WEIGHTED ? 3u : 2u) * bytes);
            bulk_g2s(buf, ka + l0, bytes, bar);
            bulk_g2s(buf + TC_KS * 8, kb + l0, bytes, bar);
            if (WEIGHTED) bulk_g2s(buf + 2 * TC_KS * 8, w + l0, bytes, bar);
        };
        if (tid == 0)
            for (int it = 0; it < 2 && it < n; ++it) issue_traj(it);
        // warps 0-7: A rows r and r + 64 of this CTA's 128, warps 8-15: B
        // columns r (and r + 64 for one SM a tile) of its BCOLS, for the
        // samples 8g .. 8g + 7, so a warp's lanes share the trajectory values
        // they load
        const bool is_b = warp >= TC_PRODUCERS / 64;
        // the partial slot of this CTA's rows of tile t
        auto slot = [&](int64_t t) { return PAIR ? 2 * (pair + t) + rank : pair + t; };
        const int r = tid & 63, g = (tid >> 6) & 3;
        SegWalk sw{u0, K};
        int trow = sw.tile / tilesC, tcol = sw.tile % tilesC;  // stepped with the tile
        int dtile = 0;  // tile of the segment being accumulated
        bool dfirst = true;
        bool failed = false;  // this thread's last wait ran out
        const int L32 = L < (int64_t)INT32_MAX ? (int)L : INT32_MAX;
        // A rows: the signed indices sa (i + oa) = +-aa of rows r and r + 64,
        // their signs in the scale: kept across stages and set at every tile
        // change for G; formed per stage for D, whose weights already hold
        // the registers (keeping them there was slower, measured)
        uint32_t aa[2];
        float sca[2];
        constexpr float kRev = 1.4629180792671596e-09f;  // 2 pi / 2^32
        auto set_rows = [&](int i0) {
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const int sja = sa * (i0 + r + 64 * v + oa);
                aa[v] = (uint32_t)(sja < 0 ? -sja : sja);
                sca[v] = sja < 0 ? -kRev : kRev;
            }
        };
        if (!WEIGHTED) set_rows(trow * SH::ROWS + (int)rank * TC_ROWS);
        for (int it = 0; it < n; ++it) {
            const int s = it % SH::STAGES;
            const uint32_t use = (uint32_t)(it / SH::STAGES);
            // stage s is free once the MMAs have consumed its previous
            // use.  Each warp waits for that itself (no producer-wide
            // barrier), so warps drift apart by at most the ring depth: a warp
            // past the wait for stage it knows every producer has finished
            // stage it - STAGES, whose trajectory slot the TMA of stage it + 2
            // reuses (it + 2 - PG_TRAJ_RING <= it - STAGES).
            if (lane == 0 && it >= SH::STAGES && !mbar_wait(bar_empty + 8 * s, (use - 1) & 1, wait_ns)) {
                *abort_flag = 1;
                atomicOr(err, kErrTimeout);
                failed = true;
            }
            // the warp stops as one: at once on a wait of its own that ran
            // out, on another warp's (the shared flag) within four stages
            if (__any_sync(0xffffffffu, failed || ((it & 3) == 0 && *abort_flag != 0))) break;
            if (tid == 0 && it + 2 < n) issue_traj(it + 2);
            if (!mbar_wait(bar_traj + 8 * (it % PG_TRAJ_RING), (uint32_t)(it / PG_TRAJ_RING) & 1, wait_ns)) {
                *abort_flag = 1;
                atomicOr(err, kErrTimeout);
                failed = true;
            }
            sw.step(it);
            if (it > 0 && sw.kc == 0) {
                if (++tcol == tilesC) {
                    tcol = 0;
                    ++trow;
                }
                if (!WEIGHTED) set_rows(trow * SH::ROWS + (int)rank * TC_ROWS);
            }
            const int l0 = sw.kc * TC_KS;
            const int j0 = tcol * PG_COLS + (int)rank * SH::BCOLS;
            const uint8_t* tbuf = smem + SH::TRAJ_OFF + (it % PG_TRAJ_RING) * PG_TRAJ_BUF;
            const int64_t* ka_s = reinterpret_cast<const int64_t*>(tbuf);
            const int64_t* kb_s = reinterpret_cast<const int64_t*>(tbuf + TC_KS * 8);
            const float2* w_s = reinterpret_cast<const float2*>(tbuf + 2 * TC_KS * 8);
            const uint32_t st = sbase + (uint32_t)s * SH::STAGE;
            const uint32_t aRH = st, aRL = st + PA_BYTES, aIH = st + 2 * PA_BYTES, aIL = st + 3 * PA_BYTES;
            const uint32_t bH = st + 4 * PA_BYTES, bL = bH + SH::B_TILE;
            if (!is_b) {
                // A rows i = i0 + r + 64 v: the signed index sa (i + oa) = +-aa,
                // its sign in the scale; the row's 8 samples in 16-byte chunk g
                // of the Ar and Ai tiles
                uint32_t klo[8], khi[8];
                float2 ww[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const uint64_t k = (uint64_t)ka_s[8 * g + e];
                    klo[e] = (uint32_t)k;
                    khi[e] = (uint32_t)(k >> 32);
                    if (WEIGHTED) {
                        ww[e] = w_s[8 * g + e];
                        ww[e].x *= wmul;
                        ww[e].y *= wmul;
                    }
                }
                float re[8], im[8];
                uint4 rh, rl, ih, il;
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                    const int row = r + 64 * v;
                    uint32_t av = aa[v];
                    float sv = sca[v];
                    if (WEIGHTED) {
                        const int sja = sa * (trow * SH::ROWS + (int)rank * TC_ROWS + row + oa);
                        av = (uint32_t)(sja < 0 ? -sja : sja);
                        sv = sja < 0 ? -kRev : kRev;
                    }
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        float2 z = phasor_top(klo[e], khi[e], 0u, av, sv);
                        if (WEIGHTED) z = cmul(z, ww[e]);
                        re[e] = z.x;
                        im[e] = z.y;
                    }
                    split8<BF16>(re, rh, rl);
                    split8<BF16>(im, ih, il);
                    st_shared_v4(aRH + sw64(row, g), rh);
                    st_shared_v4(aRL + sw64(row, g), rl);
                    st_shared_v4(aIH + sw64(row, g), ih);
                    st_shared_v4(aIL + sw64(row, g), il);
                }
            } else {
                // B columns j = j0 + r (+ 64): the phase k (j + half / 2) has the top
                // 32 bits umulhi(lo, j) + hi j + half (hi >> 1), those of
                // kq j + half (kq >> 1) mod 2^64 up to the carry out of the low
                // words (one unit of 2^-32 cycle).  Samples past L (only in a
                // tile's last chunk): A is zero there through the zero padding
                // of the weights, or B by the mask when unweighted; columns
                // past J are zero.
                const int nvalid = (!WEIGHTED && l0 + TC_KS > L32) ? L32 - l0 : TC_KS;
                const float scb = sb < 0 ? -kRev : kRev;
                uint32_t klo[8], khi[8], kc[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const uint64_t k = (uint64_t)kb_s[8 * g + e];
                    klo[e] = (uint32_t)k;
                    khi[e] = (uint32_t)(k >> 32);
                    // half-integer offsets only for D (weighted); G's are integers
                    kc[e] = (WEIGHTED && half) ? (uint32_t)((int32_t)khi[e] >> 1) : 0u;
                }
#pragma unroll
                for (int v = 0; v < SH::BCOLS / 64; ++v) {
                    if (nvalid == TC_KS && j0 + SH::BCOLS <= J)
                        pair_b_col<BF16, false, SH::BCOLS>(klo, khi, kc, j0, r + 64 * v, g, J, nvalid, scb, bH, bL);
                    else
                        pair_b_col<BF16, true, SH::BCOLS>(klo, khi, kc, j0, r + 64 * v, g, J, nvalid, scb, bH, bL);
                }
            }
            // every lane's stores are made visible to the tensor core's
            // proxy before the warp's one arrival at the MMA issuer's CTA
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) {
                if constexpr (PAIR) mbar_arrive_cluster(bar_full + 8 * s, 0);
                else mbar_arrive(bar_full + 8 * s);
            }
            if (sw.pos == 0) {
                // the MMA now has the first stage of a new segment queued:
                // drain the previous one
                if (sw.seg > 0) {
                    const int j = sw.seg - 1;
                    if (!mbar_wait(bar_acc_full, (uint32_t)j & 1, wait_ns)) {
                        atomicOr(err, kErrTimeout);
                        *abort_flag = 1;
                    }
                    __syncwarp();  // the tensor-memory loads are warp-collective
                    tc_fence_after();
                    drain_pairs<SH::BCOLS>(tmem, part + slot(dtile) * TC_TILE_FLOATS, warp, lane, dfirst);
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        if constexpr (PAIR) mbar_arrive_cluster(bar_acc_empty, 0);
                        else mbar_arrive(bar_acc_empty);
                    }
                }
                dtile = sw.tile;
                dfirst = sw.first_of_tile;
            }
        }
        // the last segment (a warp drains it as one, or not at all)
        if (sw.seg >= 0 && !__any_sync(0xffffffffu, *abort_flag != 0)) {
            const int j = sw.seg;
            const bool landed = mbar_wait(bar_acc_full, (uint32_t)j & 1, wait_ns);
            if (!landed) atomicOr(err, kErrTimeout);
            if (__all_sync(0xffffffffu, landed)) {
                tc_fence_after();
                drain_pairs<SH::BCOLS>(tmem, part + slot(dtile) * TC_TILE_FLOATS, warp, lane, dfirst);
            }
        }
        // every requested chunk has landed before the CTA goes (at most one
        // request per ring slot is open: the last PG_TRAJ_RING stages)
        if (tid == 0)
            for (int j = issued > PG_TRAJ_RING ? issued - PG_TRAJ_RING : 0; j < issued; ++j)
                if (!mbar_wait(bar_traj + 8 * (j % PG_TRAJ_RING), (uint32_t)(j / PG_TRAJ_RING) & 1, kDrainNs))
                    atomicOr(err, kErrTimeout);
    } else if (rank == 0 && lane == 0) {
        // ------------------------------------------------ MMA issuer (the tile's)
        // kind::f16, D = F32 (bit 4), A/B = F16 (0) or BF16 (1) at bits 7 and
        // 10, both K-major, N = 256 (N>>3 at bit 17), M = ROWS (M>>4 at bit 24).
        const uint32_t fmt = BF16 ? 1u : 0u;
        const uint32_t idesc =
            (1u << 4) | (fmt << 7) | (fmt << 10) | ((256u >> 3) << 17) | (((uint32_t)SH::ROWS >> 4) << 24);
        SegWalk sw{u0, K};
        int issued = 0;  // stages whose MMAs were issued
        // a test's injected stall: nothing completes bar_drain before this
        // thread's own commit, so the bounded wait runs out and no MMA issues
        if (stall && !mbar_wait(bar_drain, 0, wait_ns)) atomicOr(err, kErrTimeout);
        // [P_ac | P_ad] per BCOLS block in TMEM columns 0-255, [P_bc | P_bd] in 256-511
        const uint32_t t_r = tmem, t_i = tmem + 256;
        for (int it = 0; !stall && it < n; ++it) {
            const int s = it % SH::STAGES;
            const uint32_t use = (uint32_t)(it / SH::STAGES);
            sw.step(it);
            if (sw.pos == 0 && sw.seg >= 1 && !mbar_wait(bar_acc_empty, (uint32_t)(sw.seg - 1) & 1, wait_ns)) {
                atomicOr(err, kErrTimeout);
                break;
            }
            if (!mbar_wait(bar_full + 8 * s, use & 1, wait_ns)) {
                atomicOr(err, kErrTimeout);
                break;
            }
            ++issued;
            tc_fence_after();
            const uint32_t st = sbase + (uint32_t)s * SH::STAGE;
            const uint32_t aRH = st, aRL = st + PA_BYTES, aIH = st + 2 * PA_BYTES, aIL = st + 3 * PA_BYTES;
            const uint32_t bH = st + 4 * PA_BYTES, bL = bH + SH::B_TILE;
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                const uint32_t o = 32u * kk;  // samples 16 kk .. 16 kk + 15 of each row
#pragma unroll
                for (int q = 0; q < 3; ++q) {  // hi*hi, hi*lo, lo*hi
                    const uint32_t Ar = q == 2 ? aRL : aRH, Ai = q == 2 ? aIL : aIH, B = q == 1 ? bL : bH;
                    const uint32_t acc = (sw.pos > 0 || kk > 0 || q > 0) ? 1u : 0u;
                    if constexpr (PAIR) {
                        mma2_f16(t_r, sdesc64(Ar + o), sdesc64(B + o), idesc, acc);
                        mma2_f16(t_i, sdesc64(Ai + o), sdesc64(B + o), idesc, acc);
                    } else {
                        mma_f16(t_r, sdesc64(Ar + o), sdesc64(B + o), idesc, acc);
                        mma_f16(t_i, sdesc64(Ai + o), sdesc64(B + o), idesc, acc);
                    }
                }
            }
            if constexpr (PAIR) {
                mma2_commit_pair(bar_empty + 8 * s);
                if (sw.closes(it, n)) mma2_commit_pair(bar_acc_full);
            } else {
                mma_commit(bar_empty + 8 * s);
                if (sw.closes(it, n)) mma_commit(bar_acc_full);
            }
        }
        // no MMA may still read the stages (of either CTA) or write TMEM once
        // the tile's CTAs free it
        if (issued > 0) {
            if constexpr (PAIR) mma2_commit_pair(bar_drain);
            else mma_commit(bar_drain);
            if (!mbar_wait(bar_drain, 0, kDrainNs)) atomicOr(err, kErrTimeout);
        }
    }

    tc_fence_before();
    __syncthreads();
    // the leader has seen its MMAs complete (they read this CTA's shared
    // memory and write its TMEM) and no arrival on the other CTA is pending
    if constexpr (PAIR) cluster_sync();
    if (warp == TC_PRODUCERS / 32) {
        __syncwarp();
        tc_fence_after();
        if constexpr (PAIR) tmem_dealloc2(tmem, 512);
        else tmem_dealloc(tmem, 512);
    }
}

// out[i][c] = scale * 2^e * (sum of the partials of the tile holding output
// (i, c) in owner order); 2^e undoes the weight scaling.  A block sums a
// patch of 32 rows x 32 columns of a partial tile (column q < 128: j = 128
// tcol + q at c+(j); q >= 128: j = 128 tcol + q - 128 at c-(j)).  The owners
// (CTAs, or CTA pairs when `pairs`) holding units of tile t are c_lo..c_hi (of
// P), the last owners whose ranges start at or before the tile's first and
// last unit; owner c keeps its partial of tile t in slot c + t, or, for a
// pair, CTA h its 128 rows' partial in slot 2 (c + t) + h.  Each thread reads four
// columns of one row as a vector, the patch turns in shared memory, and
// writes run along the rows of out (the mirrored half in descending columns).
// c-(0) = c+(0) for integer offsets and is written once.
__global__ void __launch_bounds__(256) k_reduce_pair(const float* __restrict__ part, int64_t U, int64_t K, int64_t P,
                                                     bool pairs, PairGeom pg, int tilesC, float scale,
                                                     const unsigned* __restrict__ amax2, float2* __restrict__ out)
{
    __shared__ float2 patch[32][33];
    float sc = scale;
    if (amax2) sc = scale / weight_scale_inv(amax2);
    const int i0 = blockIdx.y * 32;
    const int tcol = blockIdx.x >> 3, q0 = (blockIdx.x & 7) * 32;  // tile column, first partial column
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const int tr = i0 / TC_ROWS;                   // 128-row block: tile row tr (or tr / 2 with CTA tr % 2)
    const int64_t t = (int64_t)(pairs ? tr >> 1 : tr) * tilesC + tcol;
    const int h = pairs ? tr & 1 : 0;
    const int64_t c_lo = ((t * K + 1) * P - 1) / U;
    const int64_t c_hi = ((t + 1) * K * P - 1) / U;
    const int row = (i0 % TC_ROWS) + tx;
    {
        // thread (tx, ty): row tx of the patch, partial columns q0 + 4 ty .. + 3
        const int cg = (q0 >> 2) + ty;
        float4 ar = make_float4(0.f, 0.f, 0.f, 0.f), ai = ar;
        // four partials' loads in flight at a time, added in pair order; an
        // empty range (or one past c_hi) adds zeros, which change no sum.
        // Ranges can be empty only when there are fewer units than pairs.
        constexpr int B = 4;
        const bool any_empty = U < P;
        for (int64_t c0 = c_lo; c0 <= c_hi; c0 += B) {
            float4 r[B], m[B];
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int64_t cc = c0 + b;
                const bool use =
                    cc <= c_hi && (!any_empty || unit_start(cc + 1, U, P) != unit_start(cc, U, P));
                const int64_t sl = pairs ? 2 * ((use ? cc : c_lo) + t) + h : (use ? cc : c_lo) + t;
                const float* pt = part + sl * TC_TILE_FLOATS;
                r[b] = *reinterpret_cast<const float4*>(pt + ((size_t)cg * TC_ROWS + row) * 4);
                m[b] = *reinterpret_cast<const float4*>(pt + ((size_t)(TC_COLS / 4 + cg) * TC_ROWS + row) * 4);
                if (!use) r[b] = m[b] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int b = 0; b < B; ++b) {
                ar.x += r[b].x; ar.y += r[b].y; ar.z += r[b].z; ar.w += r[b].w;
                ai.x += m[b].x; ai.y += m[b].y; ai.z += m[b].z; ai.w += m[b].w;
            }
        }
        patch[4 * ty + 0][tx] = make_float2(ar.x * sc, ai.x * sc);
        patch[4 * ty + 1][tx] = make_float2(ar.y * sc, ai.y * sc);
        patch[4 * ty + 2][tx] = make_float2(ar.z * sc, ai.z * sc);
        patch[4 * ty + 3][tx] = make_float2(ar.w * sc, ai.w * sc);
    }
    __syncthreads();
    const int q = q0 + tx;
    const bool mirrored = q >= PG_COLS;
    const int j = tcol * PG_COLS + (mirrored ? q - PG_COLS : q);
    const int off = 2 * j + pg.half;
    const int c = mirrored ? (pg.C2 - off) / 2 : (pg.C2 + off) / 2;
    const bool ok = j < pg.J && c >= 0 && c < pg.C && !(mirrored && off == 0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = i0 + ty + 8 * k;
        if (ok && i < pg.R) out[(int64_t)i * pg.C + c] = patch[tx][ty + 8 * k];
    }
}

// w'_l = w_l exp(sb i2pi (kb_l / 2) shift2) for l < L (the weight of the
// original B operand and the phase of the pairing's centre column, shift2 =
// C2 + 2 ob); the plan's buffer keeps its zero padding past L.  amax2 (zeroed
// before the launch) receives max_l |w'_l|^2 as float bits, as k_absmax2.
__global__ void k_pair_weights(const float2* __restrict__ w, const int64_t* __restrict__ kb, int64_t L, int sb,
                               int shift2, float2* __restrict__ wp, unsigned* amax2)
{
    float mx = 0.f;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L; l += (int64_t)gridDim.x * blockDim.x) {
        float2 e = phasor_q(kb[l] >> 1, shift2);
        if (sb < 0) e.y = -e.y;
        const float2 v = cmul(w[l], e);
        wp[l] = v;
        mx = fmaxf(mx, fmaf(v.x, v.x, v.y * v.y));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && isfinite(mx)) atomicMax(amax2, __float_as_uint(mx));
}

// ------------------------------------------------------------ forward H f

// The forward NUDFT (Hf)_l = (1/N) sum_n e^{+i2pi ky_l n} sum_m f[n][m]
// e^{+i2pi kx_l m} (Eq. ModDirect) as the contraction
//      P[l][m] = sum_n e^{+i2pi ky_l n} f[n][m]        (tensor cores, K = n)
// followed by the per-sample dot product y_l = (1/N) sum_m P[l][m]
// e^{+i2pi kx_l m}.  A tile is 128 samples (TMEM lanes) x 256 image columns
// m, so each thread of the epilogue owns one sample and sums its own lane's
// columns: no reduction across lanes.  A (the phases) is generated by the
// producers; B (the image, split into hi/lo and laid out exactly as a stage
// expects, k_split_image) arrives per stage by one 64 KB TMA bulk copy.
// CTA c takes the sample tiles c, c + P, ...; per tile the m-tiles in order,
// per m-tile the 32-row chunks of n.

constexpr uint32_t FW_YPART = TC_STAGES * STAGE_BYTES;  // 4 x 128 float2
constexpr uint32_t FW_BAR = FW_YPART + 4 * TC_ROWS * 8;
constexpr uint32_t FW_SMEM = FW_BAR + 128 + 1024;
static_assert(FW_SMEM <= 232448, "shared memory per CTA");
constexpr uint32_t FW_BLOCK = 2 * B_BYTES;  // one m-tile x 32-row chunk: hi then lo

// Image f (N x N, row n, column m) -> per (m-tile, n-chunk) block the B
// operand of a stage: rows m (256), K = 32 values of n as [re | im], hi and
// lo halves, 128-byte-swizzled K-major.  Rows m >= N and n >= N are zero.
// The values are scaled by 2^-e, 2^e >= max |f| (amax2 = max |f|^2), so the
// FP16 halves stay in range; k_tc_forward undoes the scale.
template <bool BF16>
__global__ void k_split_image(const float2* __restrict__ f, int N, int kchunks, const unsigned* __restrict__ amax2,
                              uint8_t* __restrict__ FB)
{
    const float wmul = weight_scale_inv(amax2);
    const int mtiles = (N + TC_COLS - 1) / TC_COLS;
    const int64_t total = (int64_t)mtiles * TC_COLS * kchunks * 4;  // (m, chunk, group of 8 n)
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(e % (mtiles * TC_COLS));  // consecutive threads: consecutive m
        const int64_t rest = e / (mtiles * TC_COLS);
        const int g = (int)(rest & 3), kc = (int)(rest >> 2);
        float re[8], im[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int n = 32 * kc + 8 * g + j;
            const float2 v = (m < N && n < N) ? f[(int64_t)n * N + m] : make_float2(0.f, 0.f);
            re[j] = v.x * wmul;
            im[j] = v.y * wmul;
        }
        uint4 rh, rl, ih, il;
        split8<BF16>(re, rh, rl);
        split8<BF16>(im, ih, il);
        const int mt = m / TC_COLS, r = m % TC_COLS;
        uint8_t* blk = FB + ((int64_t)mt * kchunks + kc) * FW_BLOCK;
        *reinterpret_cast<uint4*>(blk + sw128(r, g)) = rh;
        *reinterpret_cast<uint4*>(blk + sw128(r, 4 + g)) = ih;
        *reinterpret_cast<uint4*>(blk + B_BYTES + sw128(r, g)) = rl;
        *reinterpret_cast<uint4*>(blk + B_BYTES + sw128(r, 4 + g)) = il;
    }
}

template <bool BF16>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_tc_forward(const int64_t* __restrict__ kxq, const int64_t* __restrict__ kyq, const uint8_t* __restrict__ FB,
             const unsigned* __restrict__ amax2, int64_t L, int N, int kchunks, float scale, float2* __restrict__ y,
             int* err, unsigned long long wait_ns, int stall)
{
    scale /= weight_scale_inv(amax2);  // undoes k_split_image's 2^-e
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar_full = sbase + FW_BAR;             // TC_STAGES: A generated and B landed
    const uint32_t bar_empty = bar_full + 8 * TC_STAGES;  // TC_STAGES: stage consumed
    const uint32_t bar_acc_full = bar_empty + 8 * TC_STAGES;
    const uint32_t bar_acc_empty = bar_acc_full + 8;
    const uint32_t bar_drain = bar_acc_empty + 8;  // every MMA issued has completed
    const uint32_t misc = FW_BAR + 8 * (2 * TC_STAGES + 3);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + misc);
    float2* ypart = reinterpret_cast<float2*>(smem + FW_YPART);  // [4 column quarters][128 samples]

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int mtiles = (N + TC_COLS - 1) / TC_COLS;
    const int64_t ntiles = (L + TC_ROWS - 1) / TC_ROWS;
    const int64_t my_tiles = (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
    const int per_tile = mtiles * kchunks;
    const int n = (int)(my_tiles * per_tile);

    if (tid == 0) {
        for (int i = 0; i < TC_STAGES; ++i) {
            mbar_init(bar_full + 8 * i, TC_PRODUCERS + 1);
            mbar_init(bar_empty + 8 * i, 1);
        }
        mbar_init(bar_acc_full, 1);
        mbar_init(bar_acc_empty, TC_PRODUCERS);
        mbar_init(bar_drain, 1);
        fence_mbar_init();
    }
    if (warp == TC_PRODUCERS / 32) tmem_alloc(smem_u32(tmem_slot), 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < TC_PRODUCERS / 32) {
        // ------------------------------------------------ producers
        // A wait that runs out sets the thread's `late`; the producers decide
        // to stop together, at the OR-barrier that starts each stage, so none
        // is left alone at a named barrier of the epilogue.
        const int r = tid & 127, g = tid >> 7;  // A row (sample in the tile), group of 8 n
        int issued = 0;                          // stages whose image block thread 0 requested
        bool late = false, stopped = false;
        int64_t ka = 0;                          // ky of this thread's sample (fixed point)
        int64_t cur_tile = -1;
        float2 ysum = make_float2(0.f, 0.f);     // threads 0..127: y of sample tid over m-tiles
        // the epilogue of the segment (tile t, m-tile mt): this warp's 64 columns
        auto epilogue = [&](int64_t t, int mt) {
            __syncwarp();  // the tensor-memory loads are warp-collective
            const int lq = warp & 3, cq = warp >> 2;
            const int rs = 32 * lq + lane;
            const int64_t l = t * TC_ROWS + rs;
            const int64_t kx = l < L ? kxq[l] : 0;
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll 1
            for (int cc = 0; cc < 64; cc += 16) {
                float re[16], im[16];
                const uint32_t ta = tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(64 * cq + cc);
                tmem_ld16(ta, re);
                tmem_ld16(ta + TC_COLS, im);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float2 w = phasor_fast(kx, mt * TC_COLS + 64 * cq + cc + j);
                    acc.x = fmaf(re[j], w.x, fmaf(-im[j], w.y, acc.x));
                    acc.y = fmaf(re[j], w.y, fmaf(im[j], w.x, acc.y));
                }
            }
            ypart[cq * TC_ROWS + rs] = acc;
            producers_sync();
            if (tid < TC_ROWS) {
                const float2 a = ypart[tid], b = ypart[TC_ROWS + tid], c = ypart[2 * TC_ROWS + tid],
                             d = ypart[3 * TC_ROWS + tid];
                ysum.x += ((a.x + b.x) + c.x) + d.x;
                ysum.y += ((a.y + b.y) + c.y) + d.y;
                if (mt == mtiles - 1) {
                    const int64_t lo = t * TC_ROWS + tid;
                    if (lo < L) y[lo] = make_float2(ysum.x * scale, ysum.y * scale);
                    ysum = make_float2(0.f, 0.f);
                }
            }
        };
        int64_t seg_t = 0;  // the segment being accumulated
        int seg_mt = 0;
        for (int it = 0; it < n; ++it) {
            const int s = it % TC_STAGES;
            const uint32_t use = (uint32_t)(it / TC_STAGES);
            const int64_t t = blockIdx.x + (int64_t)(it / per_tile) * gridDim.x;
            const int rem = it % per_tile, mt = rem / kchunks, kc = rem % kchunks;
            if (tid == 0 && it >= TC_STAGES && !mbar_wait(bar_empty + 8 * s, (use - 1) & 1, wait_ns)) {
                late = true;
                atomicOr(err, kErrTimeout);
            }
            if (producers_any(late)) {  // stage s is free, or every producer stops here
                stopped = true;
                break;
            }
            const uint32_t st = sbase + (uint32_t)s * STAGE_BYTES;
            const uint32_t aH = st, aL = st + A_BYTES, bH = st + 2 * A_BYTES;
            // from here to its arrival below every producer completes the
            // stage, so the phase of bar_full[s] ends once the block lands
            if (tid == 0) {
                ++issued;
                fence_proxy_async();
                mbar_expect_tx(bar_full + 8 * s, FW_BLOCK);
                bulk_g2s(bH, FB + ((int64_t)mt * kchunks + kc) * FW_BLOCK, FW_BLOCK, bar_full + 8 * s);
            }
            if (t != cur_tile) {
                const int64_t l = t * TC_ROWS + r;
                ka = l < L ? kyq[l] : 0;
                cur_tile = t;
            }
            const bool valid = t * TC_ROWS + r < L;
            float re[8], im[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                float2 v = phasor_fast(ka, 32 * kc + 8 * g + e);
                if (!valid) v = make_float2(0.f, 0.f);
                re[e] = v.x;
                im[e] = v.y;
            }
            uint4 rh, rl, ih, il;
            split8<BF16>(re, rh, rl);
            split8<BF16>(im, ih, il);
            st_shared_v4(aH + sw128(r, g), rh);
            st_shared_v4(aH + sw128(r, 4 + g), ih);
            st_shared_v4(aL + sw128(r, g), rl);
            st_shared_v4(aL + sw128(r, 4 + g), il);
            fence_proxy_async();
            mbar_arrive(bar_full + 8 * s);
            if (kc == 0) {
                if (it > 0) {
                    // the MMA has the first stage of a new segment queued: the
                    // epilogue of the previous one
                    const int j = it / kchunks - 1;
                    if (!mbar_wait(bar_acc_full, (uint32_t)j & 1, wait_ns)) {
                        atomicOr(err, kErrTimeout);
                        late = true;  // every producer still runs the epilogue (it holds a named barrier)
                    }
                    tc_fence_after();
                    epilogue(seg_t, seg_mt);
                    tc_fence_before();
                    mbar_arrive(bar_acc_empty);
                }
                seg_t = t;
                seg_mt = mt;
            }
        }
        if (n > 0 && !stopped) {
            const int j = n / kchunks - 1;
            if (!mbar_wait(bar_acc_full, (uint32_t)j & 1, wait_ns)) {
                atomicOr(err, kErrTimeout);
                late = true;
            }
            if (!producers_any(late)) {  // the last epilogue: all producers or none
                tc_fence_after();
                epilogue(seg_t, seg_mt);
            }
        }
        // every requested image block has landed before the CTA goes (the
        // open requests are among the last TC_STAGES stages)
        if (tid == 0)
            for (int j = issued > TC_STAGES ? issued - TC_STAGES : 0; j < issued; ++j)
                if (!mbar_wait(bar_full + 8 * (j % TC_STAGES), (uint32_t)(j / TC_STAGES) & 1, kDrainNs))
                    atomicOr(err, kErrTimeout);
    } else if (lane == 0) {
        // ------------------------------------------------ MMA issuer
        const uint32_t fmt = BF16 ? 1u : 0u;
        const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
        const uint32_t idesc_neg = idesc | (1u << 13);
        const uint32_t tre = tmem, tim = tmem + TC_COLS;
        int issued = 0;  // stages whose MMAs were issued
        // a test's injected stall (as in k_tc_pair_gemm)
        if (stall && !mbar_wait(bar_drain, 0, wait_ns)) atomicOr(err, kErrTimeout);
        for (int it = 0; !stall && it < n; ++it) {
            const int s = it % TC_STAGES;
            const uint32_t use = (uint32_t)(it / TC_STAGES);
            const int kc = (it % per_tile) % kchunks;
            const int seg = it / kchunks;
            if (kc == 0 && seg >= 1 && !mbar_wait(bar_acc_empty, (uint32_t)(seg - 1) & 1, wait_ns)) {
                atomicOr(err, kErrTimeout);
                break;
            }
            if (!mbar_wait(bar_full + 8 * s, use & 1, wait_ns)) {
                atomicOr(err, kErrTimeout);
                break;
            }
            ++issued;
            tc_fence_after();
            const uint32_t st = sbase + (uint32_t)s * STAGE_BYTES;
            const uint32_t aH = st, aL = st + A_BYTES, bH = st + 2 * A_BYTES, bL = bH + B_BYTES;
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                const uint32_t oR = 32u * kk, oI = 64u + 32u * kk;
#pragma unroll
                for (int q = 0; q < 3; ++q) {  // hi*hi, hi*lo, lo*hi
                    const uint32_t A = q == 2 ? aL : aH, B = q == 1 ? bL : bH;
                    const uint32_t acc = (kc > 0 || kk > 0 || q > 0) ? 1u : 0u;
                    mma_f16(tre, sdesc(A + oR), sdesc(B + oR), idesc, acc);
                    mma_f16(tre, sdesc(A + oI), sdesc(B + oI), idesc_neg, 1u);
                    mma_f16(tim, sdesc(A + oR), sdesc(B + oI), idesc, acc);
                    mma_f16(tim, sdesc(A + oI), sdesc(B + oR), idesc, 1u);
                }
            }
            mma_commit(bar_empty + 8 * s);
            if (kc == kchunks - 1) mma_commit(bar_acc_full);
        }
        // no MMA may still read the stages or write TMEM once the CTA frees it
        if (issued > 0) {
            mma_commit(bar_drain);
            if (!mbar_wait(bar_drain, 0, kDrainNs)) atomicOr(err, kErrTimeout);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == TC_PRODUCERS / 32) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// amax2 = max_l |y_l|^2 as float bits (non-negative floats order like unsigned).
__global__ void k_absmax2(const float2* __restrict__ y, int64_t n, unsigned* amax2)
{
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = y[i];
        m = fmaxf(m, fmaf(v.x, v.x, v.y * v.y));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && isfinite(m)) atomicMax(amax2, __float_as_uint(m));
}

// The pairing geometry of G (knob SPIREC_KNOB_GRAM_SPLIT) or of D and every
// other H^H y (SPIREC_KNOB_ADJOINT_SPLIT): see PairGeom.
PairGeom pair_geom(const spirec_plan_s* p, int knob)
{
    const int N = p->N;
    PairGeom g{};
    g.R = N;
    if (knob == SPIREC_KNOB_GRAM_SPLIT) {
        g.C = 2 * N - 1;
        g.C2 = 2 * N - 2;
        g.half = 0;
        g.J = N;
    } else {
        g.C = N;
        g.C2 = N - 1;
        g.half = (N % 2 == 0) ? 1 : 0;
        g.J = g.half ? N / 2 : (N + 1) / 2;
    }
    return g;
}

// Clusters of two k_tc_pair_gemm CTAs the device runs at once (cached per
// device): the pairs a launch may spread its work over.
int pair_clusters(int* out)
{
    static int cached[64];
    int dev = 0;
    SPIREC_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) dev = 63;
    if (cached[dev] <= 0) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(2 * (kMaxCtas / 2));
        cfg.blockDim = dim3(TC_THREADS);
        cfg.dynamicSmemBytes = PairShape<true>::SMEM;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        SPIREC_CK(cudaOccupancyMaxActiveClusters(&n, (void*)k_tc_pair_gemm<false, false, true>, &cfg));
        if (n < 1) {
            set_error("the device runs no cluster of two contraction CTAs");
            return SPIREC_EUNSUPPORTED;
        }
        cached[dev] = n;
    }
    *out = cached[dev];
    return SPIREC_OK;
}

template <bool BF16, bool WEIGHTED, bool PAIR>
cudaError_t launch_pair_kernel(int64_t P, cudaStream_t stream, const int64_t* ka, const int64_t* kb, const float2* w,
                               const unsigned* amax, int64_t L, int tilesC, int oa, int sa, int sb, int half, int J,
                               int64_t K, int64_t U, float* part, int* err, unsigned long long wait_ns, int stall)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)P);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = PairShape<PAIR>::SMEM;
    cfg.stream = stream;
    cfg.attrs = PAIR ? at : nullptr;
    cfg.numAttrs = PAIR ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_tc_pair_gemm<BF16, WEIGHTED, PAIR>, ka, kb, w, amax, L, tilesC, oa, sa, sb, half,
                              J, K, U, part, err, wait_ns, stall);
}

template <bool PAIR>
cudaError_t launch_pair_any(bool bf16, int64_t P, cudaStream_t stream, const int64_t* ka, const int64_t* kb,
                            const float2* w, const unsigned* amax, int64_t L, int tilesC, int oa, int sa, int sb,
                            int half, int J, int64_t K, int64_t U, float* part, int* err, unsigned long long wait_ns,
                            int stall)
{
    if (bf16 && w)
        return launch_pair_kernel<true, true, PAIR>(P, stream, ka, kb, w, amax, L, tilesC, oa, sa, sb, half, J, K, U,
                                                    part, err, wait_ns, stall);
    if (bf16)
        return launch_pair_kernel<true, false, PAIR>(P, stream, ka, kb, w, amax, L, tilesC, oa, sa, sb, half, J, K, U,
                                                     part, err, wait_ns, stall);
    if (w)
        return launch_pair_kernel<false, true, PAIR>(P, stream, ka, kb, w, amax, L, tilesC, oa, sa, sb, half, J, K, U,
                                                     part, err, wait_ns, stall);
    return launch_pair_kernel<false, false, PAIR>(P, stream, ka, kb, w, amax, L, tilesC, oa, sa, sb, half, J, K, U,
                                                  part, err, wait_ns, stall);
}

// The paired contraction out[i][c] = scale sum_l A(l,i) B(l,c) with
// A(l,i) = exp(sa i2pi ka_l (i + oa)), B(l,c) = w_l exp(sb i2pi kb_l (c + ob)).
int tc_pair_gemm(spirec_plan p, int knob, const int64_t* ka, const int64_t* kb, const float2* w, int oa, int ob,
                 int sa, int sb, float scale, float2* out)
{
    const PairGeom pg = pair_geom(p, knob);
    int sms = 0, rc;
    if ((rc = device_sms(&sms)) != SPIREC_OK) return rc;
    const bool pairs = tc_pairs(p, knob, sms);
    const int rows = pairs ? PairShape<true>::ROWS : PairShape<false>::ROWS;
    const int64_t K = (p->L + TC_KS - 1) / TC_KS;
    const int tilesR = (pg.R + rows - 1) / rows, tilesC = (pg.J + PG_COLS - 1) / PG_COLS;
    const int64_t T = (int64_t)tilesR * tilesC;
    const int64_t U = T * K;
    if (U > (int64_t)INT32_MAX) {
        set_error("%lld contraction units exceed the kernel's 32-bit unit counters", (long long)U);
        return SPIREC_EUNSUPPORTED;
    }
    if (!w && pg.half) {
        set_error("an unweighted paired contraction takes integer offsets");
        return SPIREC_EUNSUPPORTED;
    }
    int64_t P = 0;
    if ((rc = tc_ctas(p, knob, sms, &P)) != SPIREC_OK) return rc;
    unsigned* amax = nullptr;
    const int shift2 = pg.C2 + 2 * ob;  // twice the phase offset of the centre column
    if (!w && shift2 != 0) {
        set_error("an unweighted paired contraction needs its centre at phase zero");
        return SPIREC_EUNSUPPORTED;
    }
    if (w) {
        // w' = w exp(sb i2pi kb shift2 / 2) into the plan's padded buffer
        // (its padding past L stays zero), and max |w'|^2 for the scaling
        int blocks = (int)((p->L + 255) / 256);
        if (blocks > 4 * kMaxCtas) blocks = 4 * kMaxCtas;
        amax = p->counters + C_AMAX;
        SPIREC_CK(cudaMemsetAsync(amax, 0, sizeof(unsigned), p->stream));
        k_pair_weights<<<blocks, 256, 0, p->stream>>>(w, kb, p->L, sb, shift2, p->wpair, amax);
        SPIREC_CK(cudaGetLastError());
        w = p->wpair;
        p->launches += 1;
    }
    float* part = p->kpart;
    const bool bf16 = p->precision == SPIREC_MIXED_BF16X3;
    const unsigned long long wait_ns = wait_limit_ns();
    const int stall = injected_stall(kStallContraction) ? 1 : 0;
    const cudaError_t le =
        pairs ? launch_pair_any<true>(bf16, P, p->stream, ka, kb, w, amax, p->L, tilesC, oa, sa, sb, pg.half, pg.J, K,
                                      U, part, p->dflag, wait_ns, stall)
              : launch_pair_any<false>(bf16, P, p->stream, ka, kb, w, amax, p->L, tilesC, oa, sa, sb, pg.half, pg.J,
                                       K, U, part, p->dflag, wait_ns, stall);
    SPIREC_CK(le);
    const dim3 rgrid((unsigned)(tilesC * 8), (unsigned)((pg.R + 31) / 32));
    k_reduce_pair<<<rgrid, dim3(32, 8), 0, p->stream>>>(part, U, K, pairs ? P / 2 : P, pairs, pg, tilesC, scale,
                                                        amax, out);
    SPIREC_CK(cudaGetLastError());
    p->launches += 2;
    return SPIREC_OK;
}

}  // namespace

int launch_forward_tc(spirec_plan p, const float2* x, float2* yout)
{
    const int N = p->N;
    const int kchunks = (N + TC_KS - 1) / TC_KS;
    const int mtiles = (N + TC_COLS - 1) / TC_COLS;
    const size_t fb_bytes = (size_t)mtiles * kchunks * FW_BLOCK;
    if (!p->fsplit || p->fsplit_bytes < fb_bytes) {
        set_error("plan has no split-image buffer for the forward contraction");
        return SPIREC_ESTATE;
    }
    const bool bf16 = p->precision == SPIREC_MIXED_BF16X3;
    unsigned* amax = p->counters + C_AMAX;
    {
        const int64_t NN = (int64_t)N * N;
        SPIREC_CK(cudaMemsetAsync(amax, 0, sizeof(unsigned), p->stream));
        int blocks = (int)((NN + 255) / 256);
        if (blocks > 4 * kMaxCtas) blocks = 4 * kMaxCtas;
        k_absmax2<<<blocks, 256, 0, p->stream>>>(x, NN, amax);
        SPIREC_CK(cudaGetLastError());
        const int64_t total = (int64_t)mtiles * TC_COLS * kchunks * 4;
        blocks = (int)((total + 255) / 256);
        if (blocks > 8 * kMaxCtas) blocks = 8 * kMaxCtas;
        if (bf16)
            k_split_image<true><<<blocks, 256, 0, p->stream>>>(x, N, kchunks, amax, p->fsplit);
        else
            k_split_image<false><<<blocks, 256, 0, p->stream>>>(x, N, kchunks, amax, p->fsplit);
        SPIREC_CK(cudaGetLastError());
    }
    int dev = 0, sms = 0;
    SPIREC_CK(cudaGetDevice(&dev));
    SPIREC_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t ntiles = (p->L + TC_ROWS - 1) / TC_ROWS;
    int64_t P = sms < kMaxCtas ? sms : kMaxCtas;
    if (P > ntiles) P = ntiles;
    const float scale = 1.0f / (float)N;
    if (bf16)
        k_tc_forward<true><<<(unsigned)P, TC_THREADS, FW_SMEM, p->stream>>>(p->kxq, p->kyq, p->fsplit, amax, p->L,
                                                                           N, kchunks, scale, yout, p->dflag,
                                                                           wait_limit_ns(),
                                                                           injected_stall(kStallContraction) ? 1 : 0);
    else
        k_tc_forward<false><<<(unsigned)P, TC_THREADS, FW_SMEM, p->stream>>>(p->kxq, p->kyq, p->fsplit, amax,
                                                                            p->L, N, kchunks, scale, yout, p->dflag,
                                                                            wait_limit_ns(),
                                                                            injected_stall(kStallContraction) ? 1 : 0);
    SPIREC_CK(cudaGetLastError());
    p->launches += 3;
    return SPIREC_OK;
}

size_t fsplit_bytes_tc(int N, int precision)
{
    if (precision == SPIREC_FP32) return 0;
    const size_t kchunks = (size_t)(N + TC_KS - 1) / TC_KS, mtiles = (size_t)(N + TC_COLS - 1) / TC_COLS;
    return mtiles * kchunks * FW_BLOCK;
}

size_t kpart_floats_tc(int N, int64_t, int precision)
{
    if (precision == SPIREC_FP32) return 0;
    // slots c + t < P + T for P CTAs and T one-SM tiles, 2 (c + t) + h <
    // 2 (P + T) for P pairs and T pair tiles; G (N rows, N paired columns)
    // has the most tiles
    const size_t cols = (size_t)((N + PG_COLS - 1) / PG_COLS);
    const size_t T1 = (size_t)((N + TC_ROWS - 1) / TC_ROWS) * cols;
    const size_t T2 = 2 * (size_t)((N + 2 * TC_ROWS - 1) / (2 * TC_ROWS)) * cols;
    return ((size_t)kMaxCtas + (T1 > T2 ? T1 : T2)) * TC_TILE_FLOATS;
}

int tc_setup_attributes()
{
    constexpr int S1 = PairShape<false>::SMEM, S2 = PairShape<true>::SMEM;
    SPIREC_CK(cudaFuncSetAttribute(k_tc_pair_gemm<false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, S1));
    SPIREC_CK(cudaFuncSetAttribute(k_tc_pair_gemm<false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, S1));
    SPIREC_CK(cudaFuncSetAttribute(k_tc_pair_gemm<true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, S1));
    SPIREC_CK(cudaFuncSetAttribute(k_tc_pair_gemm<true, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, S1));
    SPIREC_CK(cudaFuncSetAttribute(k_tc_pair_gemm<false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, S2));
    SPIREC_CK(cudaFuncSetAttribute(k_tc_pair_gemm<false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, S2));
    SPIREC_CK(cudaFuncSetAttribute(k_tc_pair_gemm<true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, S2));
    SPIREC_CK(cudaFuncSetAttribute(k_tc_pair_gemm<true, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, S2));
    SPIREC_CK(cudaFuncSetAttribute(k_tc_forward<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, FW_SMEM));
    SPIREC_CK(cudaFuncSetAttribute(k_tc_forward<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, FW_SMEM));
    return SPIREC_OK;
}

int launch_gram_tc(spirec_plan p)
{
    const int N = p->N;
    // G[u][v+N-1] = (1/N^2) sum_l exp(i2pi kx_l u) exp(i2pi ky_l v), v = +-j
    return tc_pair_gemm(p, SPIREC_KNOB_GRAM_SPLIT, p->kxq, p->kyq, nullptr, 0, -(N - 1), +1, +1,
                        1.0f / ((float)N * (float)N), p->G);
}

int launch_adjoint_tc(spirec_plan p, const float2* y, float2* x)
{
    const int N = p->N;
    // x[n][m] = (1/N) sum_l exp(-i2pi ky_l n) y_l exp(-i2pi kx_l m)
    return tc_pair_gemm(p, SPIREC_KNOB_ADJOINT_SPLIT, p->kyq, p->kxq, y, 0, 0, -1, -1, 1.0f / (float)N, x);
}

// The tile shape of a contraction (knob SPIREC_KNOB_GRAM_TILE or
// SPIREC_KNOB_ADJOINT_TILE beside the split knob): the tuned value (1: one SM
// a tile of 128 rows, 2: CTA pairs, tiles of 256 rows), else pairs, except
// where pair tiles would pad more than 256 output rows further than one-SM
// tiles do (R = 384, 640, ...: the pair's last tile half empty).  Measured at
// L = 131072: R = 384, G 0.37 ms one SM a tile, 0.44 ms pairs; R = 512,
// 0.63 and 0.58 ms.
bool tc_pairs(spirec_plan p, int knob, int sms)
{
    const int tile_knob = knob == SPIREC_KNOB_GRAM_SPLIT ? SPIREC_KNOB_GRAM_TILE : SPIREC_KNOB_ADJOINT_TILE;
    const int tuned = tune_lookup(tile_knob, p, sms);
    if (tuned == 1) return false;
    if (tuned == 2) return true;
    const int R = pair_geom(p, knob).R;
    const int pad2 = (R + 2 * TC_ROWS - 1) / (2 * TC_ROWS) * (2 * TC_ROWS), pad1 = (R + TC_ROWS - 1) / TC_ROWS * TC_ROWS;
    return R <= 2 * TC_ROWS || pad2 == pad1;
}

// The stream-K CTA count: the tuned value of the shape, else one CTA per SM
// (at most kMaxCtas), rounded down to even (at least 2) for CTA pairs; never
// more owners (CTAs or pairs) than work units or, for pairs, than the device
// runs at once, and the partial slots must fit the split-K buffer (c + t <
// P + T, or 2 (c + t) + h < 2 (P / 2 + T) for pairs).
int tc_ctas(spirec_plan p, int knob, int sms, int64_t* out)
{
    const PairGeom pg = pair_geom(p, knob);
    const bool pairs = tc_pairs(p, knob, sms);
    const int rows = pairs ? PairShape<true>::ROWS : PairShape<false>::ROWS;
    const int64_t K = (p->L + TC_KS - 1) / TC_KS;
    const int64_t T = (int64_t)((pg.R + rows - 1) / rows) * ((pg.J + PG_COLS - 1) / PG_COLS);
    const int64_t U = T * K;
    const int per = pairs ? 2 : 1;  // CTAs an owner
    int64_t Q = (sms < kMaxCtas ? sms : kMaxCtas) / per;
    const int tuned = tune_lookup(knob, p, sms);
    if (tuned > 0 && tuned / per < Q) Q = tuned / per > 0 ? tuned / per : 1;
    if (pairs) {
        int clusters = 0, rc;
        if ((rc = pair_clusters(&clusters)) != SPIREC_OK) return rc;
        if (Q > clusters) Q = clusters;
    }
    if (Q > U) Q = U;
    const int64_t cap = (int64_t)(p->kpart_bytes / (TC_TILE_FLOATS * sizeof(float))) / per;
    if (Q + T > cap) Q = cap - T;
    if (Q < 1) {
        set_error("partial buffer too small for %lld tiles", (long long)T);
        return SPIREC_EUNSUPPORTED;
    }
    *out = per * Q;
    return SPIREC_OK;
}

}  // namespace spirec
