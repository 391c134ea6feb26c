// cg_device.cuh -- per-pixel bodies of the line search and of the gradient/
// update step (see cg.cu for the math), shared by the stand-alone kernels and
// the persistent CG loop.  Iterates are read with ld.global.cg so a
// persistent kernel never sees a stale L1 line written by another block.
#pragma once

#include "internal.cuh"
#include "reduce.cuh"

namespace spirec {
namespace cgd {

__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 f2axpy(float t, float2 d, float2 f)
{
    return make_float2(fmaf(t, d.x, f.x), fmaf(t, d.y, f.y));
}
__device__ __forceinline__ float redot(float2 a, float2 b) { return fmaf(a.x, b.x, a.y * b.y); }

// Line-search terms of one pixel from its values: the right and down edges
// (Omega1, masked by has_r / has_d) and the pixel (Omega0).
// num += lambda b(|x|) Re(conj(x) w), den += lambda b(|x|) |w|^2 with x = z + t w.
// KIND >= 0 fixes phi at compile time (penalty.cuh).
template <int KIND = -1>
__device__ __forceinline__ void ls_terms(float2 fp, float2 dp, float2 fr, float2 dr, float2 fd, float2 dd,
                                         bool has_r, bool has_d, const Reg& reg, float tf, float& num,
                                         float& den)
{
    if (reg.lambda1 != 0.f) {
        {
            const float2 w = f2sub(dr, dp);
            const float2 x = f2axpy(tf, w, f2sub(fr, fp));
            const float b = has_r ? reg.lambda1 * phi_weight_k<KIND>(reg.kind, reg.alpha1, redot(x, x)) : 0.f;
            num = fmaf(b, redot(x, w), num);
            den = fmaf(b, redot(w, w), den);
        }
        {
            const float2 w = f2sub(dd, dp);
            const float2 x = f2axpy(tf, w, f2sub(fd, fp));
            const float b = has_d ? reg.lambda1 * phi_weight_k<KIND>(reg.kind, reg.alpha1, redot(x, x)) : 0.f;
            num = fmaf(b, redot(x, w), num);
            den = fmaf(b, redot(w, w), den);
        }
    }
    if (reg.lambda0 != 0.f) {
        const float2 x = f2axpy(tf, dp, fp);
        const float b = reg.lambda0 * phi_weight_k<KIND>(reg.kind, reg.alpha0, redot(x, x));
        num = fmaf(b, redot(x, dp), num);
        den = fmaf(b, redot(dp, dp), den);
    }
}

// Line-search sums at step t for pixel p of the global iterates (clamped
// neighbours, masked terms).  All loads first.
template <int KIND = -1>
__device__ __forceinline__ void ls_pixel(int p, int N, const float2* f, const float2* d, const Reg& reg,
                                         float tf, float& num, float& den)
{
    const int n = p / N, m = p - n * N;
    const bool has_r = m + 1 < N, has_d = n + 1 < N;
    const int pr = has_r ? p + 1 : p, pd = has_d ? p + N : p;
    const float2 fp = __ldcg(f + p), dp = __ldcg(d + p), fr = __ldcg(f + pr), dr = __ldcg(d + pr);
    const float2 fd = __ldcg(f + pd), dd = __ldcg(d + pd);
    ls_terms<KIND>(fp, dp, fr, dr, fd, dd, has_r, has_d, reg, tf, num, den);
}

// t_{j+1} from t_j and the grid sums (majorize-minimize step; t stays when
// the curvature is not positive).
__device__ __forceinline__ double ls_next(double t, double q1, double q2, double num, double den)
{
    const double h1 = q1 + 2.0 * q2 * t + num;
    const double c = 2.0 * q2 + den;
    return c > 0.0 ? t - h1 / c : t;
}

// ls_next in float-float arithmetic (the persistent loop, where the step sits
// between a grid synchronisation and the next phase of every block).
__device__ __forceinline__ FF ls_next_ff(FF t, FF q1, FF q2, FF num, FF den)
{
    const FF q2x2 = ff_twice(q2);
    const FF h1 = ff_add(ff_add(q1, ff_mul(q2x2, t)), num);
    const FF c = ff_add(q2x2, den);
    return c.hi > 0.f ? ff_add(t, ff_neg(ff_div_pos(h1, c))) : t;
}

// Gradient at a pixel from its values: g = 2 res + grad R(f), res = T f - D
// the data term's residual in the image domain, and its share rv of R (right
// and down edges, the pixel).  An edge from p to q with z = f_q - f_p adds
// +psi(z) at q and -psi(z) at p, psi(z) = b(|z|) z.  Masked neighbours carry
// the centre value (z = 0).
template <int KIND = -1>
__device__ __forceinline__ float2 grad_at(float2 fc, float2 fu, float2 fl, float2 fdn, float2 fr, float2 rs,
                                          bool has_u, bool has_l, bool has_d, bool has_r, const Reg& reg, float& rv)
{
    float2 gp = make_float2(2.f * rs.x, 2.f * rs.y);
    rv = 0.f;
    if (reg.lambda1 != 0.f) {
        const float l1 = reg.lambda1;
        const float2 zu = f2sub(fc, fu), zl = f2sub(fc, fl), zd = f2sub(fdn, fc), zr = f2sub(fr, fc);
        const float ru = redot(zu, zu), rl = redot(zl, zl), rd = redot(zd, zd), rr = redot(zr, zr);
        float wd, vd, wr, vr;
        phi_wv_k<KIND>(reg.kind, reg.alpha1, rd, wd, vd);
        phi_wv_k<KIND>(reg.kind, reg.alpha1, rr, wr, vr);
        const float bu = has_u ? l1 * phi_weight_k<KIND>(reg.kind, reg.alpha1, ru) : 0.f;
        const float bl = has_l ? l1 * phi_weight_k<KIND>(reg.kind, reg.alpha1, rl) : 0.f;
        const float bd = has_d ? l1 * wd : 0.f;
        const float br = has_r ? l1 * wr : 0.f;
        gp = f2axpy(bu, zu, gp);
        gp = f2axpy(bl, zl, gp);
        gp = f2axpy(-bd, zd, gp);
        gp = f2axpy(-br, zr, gp);
        rv = (has_d ? l1 * vd : 0.f) + (has_r ? l1 * vr : 0.f);
    }
    if (reg.lambda0 != 0.f) {
        const float r2 = redot(fc, fc);
        float w0, v0;
        phi_wv_k<KIND>(reg.kind, reg.alpha0, r2, w0, v0);
        gp = f2axpy(reg.lambda0 * w0, fc, gp);
        rv = fmaf(reg.lambda0, v0, rv);
    }
    return gp;
}

// Gradient and step at pixel p.  Unless FIRST: f_out = f_in + t d,
// res += t Td (res = T f - D: T is linear and D fixed, so the residual moves
// by t T d; carrying it, rather than T f, keeps its FP32 rounding relative to
// the residual instead of to D, of which it is a small fraction near the
// minimum).  g = 2 res + grad R(f); per-thread sums
//   a[0] <g,g>, a[1] Re<g, g_old>, a[2] Re<g, d>, a[3] R(f), a[4] Re<f, D>, a[5] Re<f, res>.
// All loads first (clamped neighbours, masked terms).
template <bool FIRST, int KIND = -1>
__device__ __forceinline__ void update_pixel(int p, int N, const float2* f_in, float2* f_out,
                                             const float2* d, float2* res, const float2* Td,
                                             const float2* __restrict__ D, float2* g, const Reg& reg,
                                             float t, float (&a)[kUpdVals])
{
    const int n = p / N, m = p - n * N;
    const bool has_u = n > 0, has_l = m > 0, has_d = n + 1 < N, has_r = m + 1 < N;
    const int pu = has_u ? p - N : p, pl = has_l ? p - 1 : p;
    const int pd = has_d ? p + N : p, pr = has_r ? p + 1 : p;
    float2 fc = __ldcg(f_in + p), fu = __ldcg(f_in + pu), fl = __ldcg(f_in + pl);
    float2 fdn = __ldcg(f_in + pd), fr = __ldcg(f_in + pr);
    float2 rs = __ldcg(res + p);
    const float2 dv = __ldg(D + p);
    float2 dc = make_float2(0.f, 0.f), gold = dc;
    if (!FIRST) {
        dc = __ldcg(d + p);
        const float2 du = __ldcg(d + pu), dl = __ldcg(d + pl), ddn = __ldcg(d + pd), dr = __ldcg(d + pr);
        const float2 tdv = __ldcg(Td + p);
        gold = __ldcg(g + p);
        fc = f2axpy(t, dc, fc);
        fu = f2axpy(t, du, fu);
        fl = f2axpy(t, dl, fl);
        fdn = f2axpy(t, ddn, fdn);
        fr = f2axpy(t, dr, fr);
        rs = f2axpy(t, tdv, rs);
        res[p] = rs;
        f_out[p] = fc;
    }
    float rv;
    const float2 gp = grad_at<KIND>(fc, fu, fl, fdn, fr, rs, has_u, has_l, has_d, has_r, reg, rv);
    a[0] += redot(gp, gp);
    if (!FIRST) {
        a[1] += redot(gp, gold);
        a[2] += redot(gp, dc);
    }
    a[3] += rv;
    a[4] += redot(fc, dv);
    a[5] += redot(fc, rs);
    g[p] = gp;
}

// Scalars after an update: J = ||s||^2 - 2 Re<f,D> + Re<f,T f> + R
// = ||s||^2 - Re<f,D> + Re<f,res> + R (T f = res + D) and the
// Polak-Ribiere beta = max(0, (<g,g> - Re<g,g_old>) / <g_old,g_old>), set to
// 0 when Re<g, -g + beta d> >= 0 (restart) or on the first gradient.
__device__ __forceinline__ void update_finish(const double* s, double ss, double gg_old,
                                              bool first, double* J, double* beta)
{
    *J = ss - s[4] + s[5] + s[3];
    double b = 0.0;
    if (!first) {
        b = gg_old > 0.0 ? (s[0] - s[1]) / gg_old : 0.0;
        if (b < 0.0) b = 0.0;
        if (-s[0] + b * s[2] >= 0.0) b = 0.0;
    }
    *beta = b;
}

}  // namespace cgd
}  // namespace spirec
