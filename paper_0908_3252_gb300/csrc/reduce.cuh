// reduce.cuh -- deterministic block and grid reductions without FP64 ALU work.
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so sums that must
// keep more than FP32 precision are carried as float-float pairs (hi + lo,
// Knuth's TwoSum; no multiplications, so FMA contraction cannot break it).
// Each thread sums its few products in FP32 and each warp its 32 threads in
// FP32 (a 5-level tree); warps, blocks and the grid combine in float-float.
// The last block of a grid to finish (ticket from an atomic counter, no
// waiting) sums the per-block pairs in index order, so the result never
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

// Block totals of K per-thread FP32 values; valid in thread 0 only.
// Contains __syncthreads(); call from all threads of the block.
template <int K>
__device__ __forceinline__ void block_partial(float (&v)[K], FF (&out)[K])
{
    __shared__ float ws[32][K];
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
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            FF acc{ws[0][k], 0.f};
            for (int w = 1; w < nw; ++w) acc = ff_add(acc, FF{ws[w][k], 0.f});
            out[k] = acc;
        }
    }
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

// Grid totals of K values from n block partials, read past L1 in index order
// (float-float throughout); valid in thread 0 only.
template <int K>
__device__ __forceinline__ void sum_parts_ff(const float2* parts, int stride, int n, FF (&tot)[K])
{
    __shared__ FF ws[32][K];
    FF acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = FF{0.f, 0.f};
    for (int i = threadIdx.x; i < n; i += blockDim.x)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float2 p = __ldcg(parts + k * stride + i);
            acc[k] = ff_add(acc[k], FF{p.x, p.y});
        }
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            FF other;
            other.hi = __shfl_down_sync(0xffffffffu, acc[k].hi, o);
            other.lo = __shfl_down_sync(0xffffffffu, acc[k].lo, o);
            acc[k] = ff_add(acc[k], other);
        }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) ws[warp][k] = acc[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            FF a = ws[0][k];
            for (int w = 1; w < nw; ++w) a = ff_add(a, ws[w][k]);
            tot[k] = a;
        }
    }
}

}  // namespace spirec
