// reduce.cuh -- deterministic block and grid reductions in FP64.
//
// Threads accumulate a few products in FP32, blocks combine them in FP64 with
// a fixed shuffle tree, and the last block of a grid to finish (ticket from an
// atomic counter, no waiting) sums the per-block partials in index order.  The
// result therefore never depends on which block ran first.
#pragma once

namespace spirec {

// Sum over the block; the result is returned to every thread.  Contains
// __syncthreads(); call from all threads.  blockDim.x <= 1024, multiple of 32.
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double ws[32];
    __shared__ double total;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) ws[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        double w = lane < nw ? ws[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
        if (lane == 0) total = w;
    }
    __syncthreads();
    return total;
}

// True in every thread of the last block of the grid to arrive.  The caller
// has written its block partial (thread 0) before the call.
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

// Sum of n block partials, read past L1, in a fixed order; every thread gets it.
__device__ __forceinline__ double sum_parts(const double* part, int n)
{
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += __ldcg(part + i);
    return block_sum(v);
}

}  // namespace spirec
