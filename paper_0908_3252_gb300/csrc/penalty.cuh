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

// phi(r); the hyperbolic form uses sqrt(a^2+r^2) - a = r^2 / (sqrt(a^2+r^2) + a).
__device__ __forceinline__ float phi_value(int kind, float alpha, float r2)
{
    if (kind == SPIREC_PHI_HUBER)
        return r2 <= alpha * alpha ? r2 : 2.f * alpha * sqrtf(r2) - alpha * alpha;
    if (kind == SPIREC_PHI_HYPERBOLIC) return 2.f * alpha * r2 / (sqrtf(fmaf(alpha, alpha, r2)) + alpha);
    return r2;
}

}  // namespace spirec
