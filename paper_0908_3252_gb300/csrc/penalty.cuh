// penalty.cuh -- the edge-preserving penalties of section 3.3 in FP32.
//
// phi acts on the modulus r = |z| of a complex pixel difference (or pixel);
// b(r) = phi'(r) / r is the weight of the half-quadratic majorant and of the
// gradient psi(z) = b(|z|) z.  Both are evaluated from r^2.
#pragma once

#include "../../include/spirec.h"

namespace spirec {

__device__ __forceinline__ float phi_weight(int kind, float alpha, float r2)
{
    if (kind == SPIREC_PHI_HUBER) return r2 <= alpha * alpha ? 2.f : 2.f * alpha * rsqrtf(r2);
    if (kind == SPIREC_PHI_HYPERBOLIC) return 2.f * alpha * rsqrtf(fmaf(alpha, alpha, r2));
    return 2.f;
}

// e(r) = (phi''(r) - b(r)) / r^2, the coefficient of the rank-one part of
// the Hessian of phi(|z|) in (Re z, Im z): b(r) I + e(r) z z^T.  Closed forms,
// finite at r = 0: Huber 0 for r <= alpha and -2 alpha / r^3 beyond;
// hyperbolic -2 alpha / (alpha^2 + r^2)^(3/2); quadratic 0.
__device__ __forceinline__ float phi_curv_e(int kind, float alpha, float r2)
{
    if (kind == SPIREC_PHI_HUBER) {
        if (r2 <= alpha * alpha) return 0.f;
        const float rs = rsqrtf(r2);
        return -2.f * alpha * rs * rs * rs;
    }
    if (kind == SPIREC_PHI_HYPERBOLIC) {
        const float rs = rsqrtf(fmaf(alpha, alpha, r2));
        return -2.f * alpha * rs * rs * rs;
    }
    return 0.f;
}

// phi(r); the hyperbolic form uses sqrt(a^2+r^2) - a = r^2 / (sqrt(a^2+r^2) + a).
__device__ __forceinline__ float phi_value(int kind, float alpha, float r2)
{
    if (kind == SPIREC_PHI_HUBER)
        return r2 <= alpha * alpha ? r2 : 2.f * alpha * sqrtf(r2) - alpha * alpha;
    if (kind == SPIREC_PHI_HYPERBOLIC) return 2.f * alpha * r2 / (sqrtf(fmaf(alpha, alpha, r2)) + alpha);
    return r2;
}

// The same with phi fixed at compile time (KIND >= 0), so a per-pixel loop
// runs only its own phi; KIND < 0 falls back to the run-time choice.
template <int KIND>
__device__ __forceinline__ float phi_weight_k(int kind, float alpha, float r2)
{
    if constexpr (KIND < 0) return phi_weight(kind, alpha, r2);
    else if constexpr (KIND == SPIREC_PHI_HUBER) return r2 <= alpha * alpha ? 2.f : 2.f * alpha * rsqrtf(r2);
    else if constexpr (KIND == SPIREC_PHI_HYPERBOLIC) return 2.f * alpha * rsqrtf(fmaf(alpha, alpha, r2));
    else return 2.f;
}

// b(r) and phi(r) together, one reciprocal square root for both:
// Huber, r = r2 rsqrt(r2) in the linear part; hyperbolic, s = sqrt(a^2 + r^2)
// from its rsqrt and phi = 2 a r^2 / (s + a) by a fast division (a few ulp).
template <int KIND>
__device__ __forceinline__ void phi_wv_k(int kind, float alpha, float r2, float& w, float& v)
{
    if constexpr (KIND < 0) {
        w = phi_weight(kind, alpha, r2);
        v = phi_value(kind, alpha, r2);
    } else if constexpr (KIND == SPIREC_PHI_HUBER) {
        const float rs = rsqrtf(r2);
        const bool quad = r2 <= alpha * alpha;
        w = quad ? 2.f : 2.f * alpha * rs;
        v = quad ? r2 : fmaf(2.f * alpha, r2 * rs, -alpha * alpha);
    } else if constexpr (KIND == SPIREC_PHI_HYPERBOLIC) {
        const float q = fmaf(alpha, alpha, r2), rs = rsqrtf(q);
        w = 2.f * alpha * rs;
        v = __fdividef(2.f * alpha * r2, fmaf(q, rs, alpha));
    } else {
        w = 2.f;
        v = r2;
    }
}

}  // namespace spirec
