// fft_reg.cuh -- 16- and 32-point DFTs held entirely in one thread's
// registers, the building blocks of the warp-level four-step FFTs (512 points
// in the persistent loop, cg_loop.cu; 1024 points in the column pass of the
// stand-alone kernels for M >= 2048, fft.cu): a DFT over each lane's
// registers, a twiddle multiply, one exchange through shared memory inside
// the warp, and a DFT over the registers again.
//
// Radix-2 in registers, every index a compile-time constant (the loops are
// fully unrolled), so no data moves between stages.  w = exp(-2 pi i / 32)
// forward, its conjugate inverse; twiddles w^m with m < 16 are the exact
// values cos(2 pi m / 32), sin(2 pi m / 32) rounded once to FP32.
#pragma once

namespace spirec {
namespace freg {

constexpr float kC1 = 0.98078528040323043f;  // cos(pi/16)
constexpr float kC2 = 0.92387953251128674f;  // cos(2 pi/16)
constexpr float kC3 = 0.83146961230254524f;  // cos(3 pi/16)
constexpr float kC4 = 0.70710678118654752f;  // cos(4 pi/16)
constexpr float kS1 = 0.19509032201612827f;  // sin(pi/16)
constexpr float kS2 = 0.38268343236508977f;  // sin(2 pi/16)
constexpr float kS3 = 0.55557023301960222f;  // sin(3 pi/16)

__host__ __device__ constexpr float cos32(int m)
{
    constexpr float c[16] = {1.f, kC1, kC2, kC3, kC4, kS3, kS2, kS1, 0.f, -kS1, -kS2, -kS3, -kC4, -kC3, -kC2, -kC1};
    return c[m];
}
__host__ __device__ constexpr float sin32(int m)
{
    constexpr float s[16] = {0.f, kS1, kS2, kS3, kC4, kC3, kC2, kC1, 1.f, kC1, kC2, kC3, kC4, kS3, kS2, kS1};
    return s[m];
}

__host__ __device__ constexpr int bitrev5(int r)
{
    return ((r & 1) << 4) | ((r & 2) << 2) | (r & 4) | ((r & 8) >> 2) | ((r & 16) >> 4);
}

__device__ __forceinline__ float2 add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// v * w^m (forward) or v * conj(w)^m (INV), m < 16.
template <bool INV, int M>
__device__ __forceinline__ float2 mulw(float2 v)
{
    if constexpr (M == 0) {
        return v;
    } else if constexpr (M == 8) {  // w^8 = -i
        return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
    } else {
        constexpr float c = cos32(M), s = INV ? sin32(M) : -sin32(M);
        return make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.y, c, v.x * s));
    }
}

// ------------------------------------------------------- 32-point DFT

// One radix-2 decimation-in-frequency stage of half-span SPAN.
template <bool INV, int SPAN, bool HALF>
__device__ __forceinline__ void dif_stage(float2 (&x)[32])
{
#pragma unroll
    for (int b = 0; b < 32; b += 2 * SPAN) {
#pragma unroll
        for (int i = 0; i < SPAN; ++i) {
            const float2 a = x[b + i];
            if constexpr (HALF) {  // the upper half is zero
                x[b + i + SPAN] = a;
            } else {
                x[b + i] = add(a, x[b + i + SPAN]);
                x[b + i + SPAN] = sub(a, x[b + i + SPAN]);
            }
        }
    }
}

// The twiddles of a DIF stage (applied after its butterflies), split out so
// that the constant exponent is a template argument.
template <bool INV, int SPAN, int I>
__device__ __forceinline__ void dif_twiddle_row(float2 (&x)[32])
{
    if constexpr (I < SPAN) {
#pragma unroll
        for (int b = 0; b < 32; b += 2 * SPAN) x[b + I + SPAN] = mulw<INV, I * (16 / SPAN)>(x[b + I + SPAN]);
        dif_twiddle_row<INV, SPAN, I + 1>(x);
    }
}

// Natural order in, bit-reversed out: X[k] ends in x[bitrev5(k)].  HALF_IN:
// x[16..31] are zero on entry (not read).
template <bool INV, bool HALF_IN = false>
__device__ __forceinline__ void dft32_dif(float2 (&x)[32])
{
    dif_stage<INV, 16, HALF_IN>(x);
    dif_twiddle_row<INV, 16, 0>(x);
    dif_stage<INV, 8, false>(x);
    dif_twiddle_row<INV, 8, 0>(x);
    dif_stage<INV, 4, false>(x);
    dif_twiddle_row<INV, 4, 0>(x);
    dif_stage<INV, 2, false>(x);
    dif_twiddle_row<INV, 2, 0>(x);
    dif_stage<INV, 1, false>(x);
}

// ------------------------------------------------------- 16-point DFTs
// Radix-2 forms over 16 registers; w16^m = w^(2m).

__host__ __device__ constexpr int bitrev4(int r)
{
    return ((r & 1) << 3) | ((r & 2) << 1) | ((r & 4) >> 1) | ((r & 8) >> 3);
}

template <int SPAN, bool HALF>
__device__ __forceinline__ void dif16_stage(float2 (&x)[16])
{
#pragma unroll
    for (int b = 0; b < 16; b += 2 * SPAN) {
#pragma unroll
        for (int i = 0; i < SPAN; ++i) {
            const float2 a = x[b + i];
            if constexpr (HALF) {
                x[b + i + SPAN] = a;
            } else {
                x[b + i] = add(a, x[b + i + SPAN]);
                x[b + i + SPAN] = sub(a, x[b + i + SPAN]);
            }
        }
    }
}

// twiddles w16^(I * 8 / SPAN) = w^(I * 16 / SPAN) on the upper halves
template <bool INV, int SPAN, int I>
__device__ __forceinline__ void twiddle16_row(float2 (&x)[16])
{
    if constexpr (I < SPAN) {
#pragma unroll
        for (int b = 0; b < 16; b += 2 * SPAN) x[b + I + SPAN] = mulw<INV, I * (16 / SPAN)>(x[b + I + SPAN]);
        twiddle16_row<INV, SPAN, I + 1>(x);
    }
}

template <int SPAN>
__device__ __forceinline__ void dit16_stage(float2 (&x)[16])
{
#pragma unroll
    for (int b = 0; b < 16; b += 2 * SPAN) {
#pragma unroll
        for (int i = 0; i < SPAN; ++i) {
            const float2 a = x[b + i], c = x[b + i + SPAN];
            x[b + i] = add(a, c);
            x[b + i + SPAN] = sub(a, c);
        }
    }
}

// Natural order in, bit-reversed out: X[k] ends in x[bitrev4(k)].
template <bool INV, bool HALF_IN = false>
__device__ __forceinline__ void dft16_dif(float2 (&x)[16])
{
    dif16_stage<8, HALF_IN>(x);
    twiddle16_row<INV, 8, 0>(x);
    dif16_stage<4, false>(x);
    twiddle16_row<INV, 4, 0>(x);
    dif16_stage<2, false>(x);
    twiddle16_row<INV, 2, 0>(x);
    dif16_stage<1, false>(x);
}

// Bit-reversed order in (x[bitrev4(k)] holds input k), natural order out.
template <bool INV>
__device__ __forceinline__ void dft16_dit(float2 (&x)[16])
{
    dit16_stage<1>(x);
    twiddle16_row<INV, 2, 0>(x);
    dit16_stage<2>(x);
    twiddle16_row<INV, 4, 0>(x);
    dit16_stage<4>(x);
    twiddle16_row<INV, 8, 0>(x);
    dit16_stage<8>(x);
}

}  // namespace freg
}  // namespace spirec
