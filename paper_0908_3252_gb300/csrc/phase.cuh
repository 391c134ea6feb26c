// phase.cuh -- exact phase reduction for the NUDFT kernels.
//
// Every k-space coordinate is held as a 64-bit two's-complement fixed-point
// fraction of a cycle, kq = round(k * 2^64) mod 2^64.  For an integer pixel
// index or lag j, kq * j mod 2^64 is then exactly (k j mod 1) * 2^64, the
// range reduction of the phase 2 pi k j of Eq. ModDirect, with no rounding at
// any |j|.  Only the top 32 bits reach the trig call.
#pragma once

#include <stdint.h>

namespace spirec {

// exp(+i 2 pi k j) for the fixed-point k.  sincospif(x) gives sin(pi x) and
// cos(pi x); x = 2 * (phase in cycles), in [-1, 1).
__device__ __forceinline__ float2 phasor_q(int64_t kq, int j)
{
    const uint64_t th = (uint64_t)kq * (uint64_t)(int64_t)j;
    const int hi = (int)(th >> 32);
    const float x = (float)hi * 0x1p-31f;
    float sn, cs;
    sincospif(x, &sn, &cs);
    return make_float2(cs, sn);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

}  // namespace spirec
