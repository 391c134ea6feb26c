// reduce.cuh -- deterministic block and grid reductions without FP64 ALU work.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so sums are carried
// as float-float pairs (hi + lo, Knuth's TwoSum; no multiplications, so FMA
// contraction cannot break it), giving about 48 significant bits.  Threads
// accumulate a few products in FP32, blocks combine the pairs with a fixed
// shuffle tree, and the last block of a grid to finish (ticket from an atomic
// counter, no waiting) sums the per-block pairs in index order.  The result
// never depends on which block ran first.  Only the final scalars are FP64.
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

// Block-wide sums of K values; every thread receives the K totals.  Contains
// __syncthreads(); call from all threads of the block.
template <int K>
__device__ __forceinline__ void block_sum_ff(FF (&v)[K])
{
    __shared__ FF ws[32][K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            FF other;
            other.hi = __shfl_down_sync(0xffffffffu, v[k].hi, o);
            other.lo = __shfl_down_sync(0xffffffffu, v[k].lo, o);
            v[k] = ff_add(v[k], other);
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) ws[warp][k] = v[k];
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        FF acc = ws[0][k];
        for (int w = 1; w < nw; ++w) acc = ff_add(acc, ws[w][k]);
        v[k] = acc;
    }
}

// True in every thread of the last block of the grid to arrive.  The caller
// has written its block partials (thread 0) before the call.
__device__ __forceinline__ bool last_block(unsigned* counter)
{
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
        is_last = atomicAdd(counter, 1u) == nblk - 1;
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

// Writes the K block totals to parts[k * stride + block] (thread 0).
template <int K>
__device__ __forceinline__ void store_parts(const FF (&v)[K], float2* parts, int stride)
{
    if (threadIdx.x == 0) {
        const int b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
#pragma unroll
        for (int k = 0; k < K; ++k) parts[k * stride + b] = make_float2(v[k].hi, v[k].lo);
    }
}

// Grid totals of K values from n block partials, read past L1 in index order;
// every thread of the (last) block receives them.
template <int K>
__device__ __forceinline__ void sum_parts_ff(const float2* parts, int stride, int n, FF (&tot)[K])
{
#pragma unroll
    for (int k = 0; k < K; ++k) {
        FF acc{0.f, 0.f};
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const float2 p = __ldcg(parts + k * stride + i);
            acc = ff_add(acc, FF{p.x, p.y});
        }
        tot[k] = acc;
    }
    block_sum_ff<K>(tot);
}

}  // namespace spirec
