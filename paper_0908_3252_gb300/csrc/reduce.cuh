// reduce.cuh -- deterministic block and grid reductions without FP64 ALU work.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so sums that must
// keep more than FP32 precision are carried as float-float pairs (hi + lo,
// Knuth's TwoSum; no multiplications, so FMA contraction cannot break it).
// Each thread sums its few products in FP32 and each warp its 32 threads in
// FP32 (a 5-level tree); warps, blocks and the grid combine in float-float.
// The last block of a grid to finish (ticket from an atomic counter, no
// waiting) sums the per-block pairs in a fixed order, so the result never
// depends on which block ran first.  Only the final scalars are FP64.
#pragma once

namespace spirec {

struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e += a.lo + b.lo;
    const float hi = s + e;
    return FF{hi, e - (hi - s)};
}

__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.hi + (double)a.lo; }

// Float-float products and quotients for scalar work on the critical path of
// a grid synchronisation (FP64 operations have long latencies on GB300; these
// are FP32 operations).  hi + lo of the result is within a few 2^-46 of the
// exact value.
__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.hi, -a.lo}; }

__device__ __forceinline__ FF ff_twice(FF a) { return FF{2.f * a.hi, 2.f * a.lo}; }

// a * b: the product of the high parts and its exact rounding error from one
// FMA (Ogita, Rump and Oishi's TwoProduct), the cross terms added to the
// error, then Dekker's Fast2Sum.  __fmul_rn / __fadd_rn / __fsub_rn are never
// contracted into FMAs.
__device__ __forceinline__ FF ff_mul(FF a, FF b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float hi = __fadd_rn(p, e);
    return FF{hi, __fsub_rn(e, __fsub_rn(hi, p))};
}

// a / b for b > 0 (Dekker's double-length division): q0 = a.hi / b.hi in
// FP32, the remainder a - b q0 in float-float, and its quotient as the
// correction.
__device__ __forceinline__ FF ff_div_pos(FF a, FF b)
{
    const float rb = __frcp_rn(b.hi);
    const float q0 = __fmul_rn(a.hi, rb);
    const FF r = ff_add(a, ff_neg(ff_mul(b, FF{q0, 0.f})));
    const float q1 = __fmul_rn(r.hi, rb);
    const float hi = __fadd_rn(q0, q1);
    return FF{hi, __fsub_rn(q1, __fsub_rn(hi, q0))};
}

// Warp-level float-float sum (valid in lane 0).
__device__ __forceinline__ FF warp_sum_ff(FF a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        FF other;
        other.hi = __shfl_down_sync(0xffffffffu, a.hi, o);
        other.lo = __shfl_down_sync(0xffffffffu, a.lo, o);
        a = ff_add(a, other);
    }
    return a;
}

// Block totals of K per-thread FP32 values; valid in thread 0 only.
// Contains __syncthreads(); call from all threads of the block.
template <int K>
__device__ __forceinline__ void block_partial(float (&v)[K], FF (&out)[K])
{
    __shared__ float ws[32][K];
    __shared__ FF wt[K];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();  // earlier readers of ws are done
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) ws[warp][k] = v[k];
    __syncthreads();
    // warp k (k < K) adds the warp sums of value k as a float-float tree
    const int nw = (blockDim.x + 31) >> 5;
    if (warp < K) {
        FF a{lane < nw ? ws[lane][warp] : 0.f, 0.f};
        a = warp_sum_ff(a);
        if (lane == 0) wt[warp] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) out[k] = wt[k];
}

// True in every thread of the last block of the grid to arrive.  Thread 0
// has written the block partials before the call; it alone fences them and
// takes the ticket.
__device__ __forceinline__ bool last_block(unsigned* counter)
{
    __shared__ bool is_last;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
        is_last = atomicAdd(counter, 1u) == nblk - 1;
        if (is_last) __threadfence();
    }
    __syncthreads();
    return is_last;
}

// Thread 0 writes the K block totals to parts[k * stride + block].
template <int K>
__device__ __forceinline__ void store_parts(const FF (&v)[K], float2* parts, int stride)
{
    if (threadIdx.x == 0) {
        const int b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
#pragma unroll
        for (int k = 0; k < K; ++k) parts[k * stride + b] = make_float2(v[k].hi, v[k].lo);
    }
}

// Grid total of one value from n block partials (float-float, index order
// per lane, then a fixed shuffle tree); valid in lane 0 of the calling warp.
// Loads are issued eight at a time before they are added.
__device__ __forceinline__ FF warp_sum_parts(const float2* parts, int n)
{
    const int lane = threadIdx.x & 31;
    FF acc{0.f, 0.f};
    for (int base = 0; base < n; base += 32 * 8) {
        float2 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int i = base + lane + 32 * j;
            v[j] = i < n ? __ldcg(parts + i) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) acc = ff_add(acc, FF{v[j].x, v[j].y});
    }
    return warp_sum_ff(acc);
}

// Grid totals of K values from n block partials, valid in thread 0 only:
// thread t adds the partials t, t + blockDim.x, ... of each value in index
// order (the loads of a round, 4 / 2 / 1 a value for K = 1 / 2-3 / more,
// issued before they are added), then a fixed float-float tree over the
// lanes of each warp and over the warps.
// Needs K <= blockDim.x / 32.
template <int K>
__device__ __forceinline__ void sum_parts_ff(const float2* parts, int stride, int n, FF (&tot)[K])
{
    __shared__ FF ws[K][32];
    __shared__ FF wt[K];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    constexpr int J = K == 1 ? 4 : (K <= 3 ? 2 : 1);
    FF acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = FF{0.f, 0.f};
    for (int base = 0; base < n; base += J * blockDim.x) {
        float2 v[K][J];
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int i = base + threadIdx.x + j * blockDim.x;
                v[k][j] = i < n ? __ldcg(parts + k * stride + i) : make_float2(0.f, 0.f);
            }
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int j = 0; j < J; ++j) acc[k] = ff_add(acc[k], FF{v[k][j].x, v[k][j].y});
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const FF a = warp_sum_ff(acc[k]);
        if (lane == 0) ws[k][warp] = a;
    }
    __syncthreads();
    if (warp < K) {
        const FF a = warp_sum_ff(lane < nw ? ws[warp][lane] : FF{0.f, 0.f});
        if (lane == 0) wt[warp] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) tot[k] = wt[k];
}

}  // namespace spirec
