"""Truncated Newton minimisation of the criterion, in FP64 (test
infrastructure only: the tests and the benchmark's comparisons call it; it
shares no code with the CUDA path and is never called by it).

Section 5 names a Newton-like method [Bertsekas 1999] as a faster replacement
for the conjugate gradient.  The reading here is the truncated (inexact)
Newton method with a conjugate-gradient inner solver.  One outer step at the
iterate f^k:
  1. g = grad J(f^k), the C oracle's gradient (d/dRe f + i d/dIm f);
  2. the Newton direction p approximately solves  Hess J(f^k) p = -g:  n_in
     steps of linear conjugate gradient from p = 0 in the real inner product
     Re<a, b> (alpha = 0 when the curvature Re<d, Hess d> is not > 0, beta = 0
     when <r, r> is 0, the same guards as the half-quadratic inner solver);
  3. the three majorize-minimize line-search steps of the PR+ CG minimiser
     (section 3.3) along p from t = 0, and f^{k+1} = f^k + t p.

The Hessian, as a real-linear map of C^{N x N} = R^{2 N^2} in the gradient's
convention, is
    Hess J v = 2 T v + sum_e lambda_e delta_e^T Hphi(z_e) delta_e v,
with T = H^H H (applied here as the definition, the adjoint of the forward
NUDFT), z_e = delta_e f^k (f_q - f_p on the edge p -> q of Omega1, f_p on a
pixel of Omega0) and, for w in C = R^2,
    Hphi(z) w = b(r) w + e(r) z Re(conj(z) w),   r = |z|,
    b(r) = phi'(r) / r,   e(r) = (phi''(r) - b(r)) / r^2,
the Hessian of phi(|z|) in (Re z, Im z): grad phi(|z|) = b(r) z, and its
derivative adds b'(r) r zhat zhat^T with b'(r) r = phi'' - b.  e is finite at
r = 0 for the three phi (closed forms in curvature_e).  With a convex phi,
Hphi is positive semidefinite and so is Hess J.

Pinned in tests/test_oracle_newton_pins.py: phi'' against central
differences of the C oracle's phi' = r b(r); the Hessian apply against central
differences of the C oracle's gradient (itself pinned by finite differences of
J); with quadratic phi one outer step of 2 N^2 inner steps lands on the dense
normal-equation solution; J never increases; and on a strictly convex problem
the iterates reach the minimiser that the PR+ CG oracle reaches.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as O


def _redot(a, b):
    return float(np.sum(a.real * b.real + a.imag * b.imag))


def phi_weight(kind, alpha, r):
    """b(r) = phi'(r) / r, elementwise (the C oracle's phi_weight)."""
    r = np.asarray(r, np.float64)
    return np.vectorize(lambda v: O.phi_weight(kind, alpha, float(v)), otypes=[np.float64])(r)


def phi_second(kind, alpha, r):
    """phi''(r) elementwise: Huber 2 for r <= alpha and 0 beyond; hyperbolic
    2 alpha^3 / (alpha^2 + r^2)^(3/2); quadratic 2."""
    r = np.asarray(r, np.float64)
    if kind == O.PHI_HUBER:
        return np.where(r <= alpha, 2.0, 0.0)
    if kind == O.PHI_HYPERBOLIC:
        return 2.0 * alpha ** 3 / (alpha * alpha + r * r) ** 1.5
    return np.full_like(r, 2.0)


def curvature_e(kind, alpha, r):
    """e(r) = (phi''(r) - b(r)) / r^2 in closed form (finite at r = 0):
    Huber 0 for r <= alpha, -2 alpha / r^3 beyond; hyperbolic
    -2 alpha / (alpha^2 + r^2)^(3/2); quadratic 0."""
    r = np.asarray(r, np.float64)
    if kind == O.PHI_HUBER:
        return np.where(r <= alpha, 0.0, -2.0 * alpha / np.maximum(r, alpha) ** 3)
    if kind == O.PHI_HYPERBOLIC:
        return -2.0 * alpha / (alpha * alpha + r * r) ** 1.5
    return np.zeros_like(r)


def _terms(f, reg: O.Reg):
    """(lambda, alpha, z, scatter) for the right edges, the down edges and the
    pixels; scatter(out, u) adds delta^T u (u at q and -u at p for an edge)."""
    def right(out, u):
        out[:, 1:] += u
        out[:, :-1] -= u

    def down(out, u):
        out[1:, :] += u
        out[:-1, :] -= u

    def pixel(out, u):
        out += u

    return [(reg.lambda1, reg.alpha1, lambda x: x[:, 1:] - x[:, :-1], right),
            (reg.lambda1, reg.alpha1, lambda x: x[1:, :] - x[:-1, :], down),
            (reg.lambda0, reg.alpha0, lambda x: x, pixel)]


def penalty_hessian_apply(f, v, reg: O.Reg):
    """sum_e lambda_e delta_e^T Hphi(z_e) delta_e v at f."""
    f = np.asarray(f, np.complex128)
    v = np.asarray(v, np.complex128)
    out = np.zeros_like(v)
    for lam, alpha, delta, scatter in _terms(f, reg):
        if lam == 0.0:
            continue
        z, w = delta(f), delta(v)
        r = np.abs(z)
        b = phi_weight(reg.kind, alpha, r)
        e = curvature_e(reg.kind, alpha, r)
        u = lam * (b * w + e * z * (z.real * w.real + z.imag * w.imag))
        scatter(out, u)
    return out


def hessian_apply(kx, ky, f, v, reg: O.Reg):
    """Hess J(f) v = 2 H^H (H v) + the penalty Hessian at f applied to v."""
    N = f.shape[0]
    return 2.0 * O.adjoint(kx, ky, O.forward(kx, ky, v), N) + penalty_hessian_apply(f, v, reg)


def _line_terms(f, d, t, reg: O.Reg):
    """Penalty parts of h'(t) and of the majorant's curvature along d:
    sums of lambda b(|z + t w|) Re(conj(z + t w) w) and lambda b(|z + t w|) |w|^2."""
    num = den = 0.0
    for lam, alpha, delta, _ in _terms(f, reg):
        if lam == 0.0:
            continue
        x = delta(f) + t * delta(d)
        w = delta(d)
        b = lam * phi_weight(reg.kind, alpha, np.abs(x))
        num += float(np.sum(b * (x.real * w.real + x.imag * w.imag)))
        den += float(np.sum(b * (w.real * w.real + w.imag * w.imag)))
    return num, den


def line_search(kx, ky, s, f, p, reg: O.Reg, steps=3):
    """Majorize-minimize steps on h(t) = J(f + t p) from t = 0, as in the PR+ CG
    minimiser:
    t <- t - h'(t) / (2 q2 + curv(t)) while the curvature is > 0, with
    q1 = Re<p, 2 H^H (H f - s)>, q2 = ||H p||^2."""
    N = f.shape[0]
    q1 = _redot(p, 2.0 * O.adjoint(kx, ky, O.forward(kx, ky, f) - s, N))
    Hp = O.forward(kx, ky, p)
    q2 = float(np.sum(np.abs(Hp) ** 2))
    t = 0.0
    for _ in range(steps):
        num, den = _line_terms(f, p, t, reg)
        h1 = q1 + 2.0 * q2 * t + num
        c = 2.0 * q2 + den
        if c > 0.0:
            t -= h1 / c
    return t


def newton_direction(kx, ky, s, f, reg: O.Reg, inner):
    """inner linear CG steps on Hess J(f) p = -grad J(f) from p = 0."""
    g = O.gradient(kx, ky, s, f, reg)
    p = np.zeros_like(g)
    r = -g
    d = r.copy()
    rho = _redot(r, r)
    for _ in range(inner):
        q = hessian_apply(kx, ky, f, d, reg)
        dq = _redot(d, q)
        alpha = rho / dq if dq > 0.0 else 0.0
        p = p + alpha * d
        r = r - alpha * q
        rho_new = _redot(r, r)
        beta = rho_new / rho if rho > 0.0 else 0.0
        d = r + beta * d
        rho = rho_new
    return p


def solve(kx, ky, s, reg: O.Reg, x0, outer, inner):
    """outer truncated-Newton steps of inner CG steps each from x0.
    Returns (x, J_hist[outer + 1]) with J_hist[k] = J(f^k)."""
    kx = np.ascontiguousarray(kx, np.float64)
    ky = np.ascontiguousarray(ky, np.float64)
    s = np.asarray(s, np.complex128)
    f = np.array(x0, np.complex128)
    Js = [O.objective(kx, ky, s, f, reg)]
    for _ in range(outer):
        p = newton_direction(kx, ky, s, f, reg, inner)
        t = line_search(kx, ky, s, f, p, reg)
        f = f + t * p
        Js.append(O.objective(kx, ky, s, f, reg))
    return f, np.array(Js)
