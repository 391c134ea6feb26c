"""Half-quadratic minimisation of the criterion, in FP64 (test infrastructure
only: the tests and the benchmark's comparisons call it; it shares no code
with the CUDA path and is never called by it).

Section 5 names a dual (half-quadratic) optimisation [Idier 2001] as a faster
replacement for the conjugate gradient.  Its multiplicative form: for a phi
with phi(sqrt(u)) concave in u (Huber, the hyperbolic phi and the quadratic
one all are), phi(r) is the lower envelope of the parabolas
    w r^2 + psi(w),   w >= 0,   touching at w = phi'(r) / (2 r),
so J(f) = min_w K(f, w) with K(f, w) = ||s - H f||^2 + sum_e [lambda_e w_e
|z_e(f)|^2 + psi(w_e)], z_e an edge difference of Omega1 or a pixel of Omega0
(section 3.3).  For fixed weights K is quadratic in f.  One outer step:
  1. at the iterate f^k, W_e = lambda_e phi'(r_e) / (2 r_e), r_e = |z_e(f^k)|
     (lambda_e = lambda1 on edges, lambda0 on pixels);
  2. f^{k+1} = n_in steps of linear conjugate gradient on the normal
     equations of K(., W),
        A f = H^H s,  A = H^H H + sum_e W_e delta_e^H delta_e,
     started at f^k (delta_e f = z_e(f): f_q - f_p for the edge p -> q, f_p
     for a pixel).
Since K(f^k, W) = J(f^k), K(., W) >= J and conjugate gradient never raises
the quadratic it minimises, J(f^{k+1}) <= J(f^k) for any n_in >= 0.
H^H H is applied as the definition, the adjoint of the forward NUDFT of the
oracle (Eq. ModDirect), so this module checks the GPU's Toeplitz form too.

Guards, shared with the GPU: alpha = rho / Re<p, A p> only when Re<p, A p> > 0
(else 0), beta = rho' / rho only when rho > 0 (else 0).

Pinned in tests/test_oracle_pins.py: with quadratic phi one outer step of
2 N^2 inner steps solves the dense normal equations (numpy solve); the
weights make K tangent to J (equal value and gradient at f^k against the C
oracle's J and gradient, which finite differences pin) and a majorant of it
at other points; J never increases; and many outer steps reach the
minimiser that the PR+ CG oracle reaches on a strictly convex problem.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as O


def _redot(a, b):
    return float(np.sum(a.real * b.real + a.imag * b.imag))


def _w(kind, alpha, lam, z):
    """lam * phi'(r) / (2 r) per element of z (r = |z|), from the C oracle's
    phi'(r) / r."""
    r = np.abs(z).ravel()
    b = np.array([O.phi_weight(kind, alpha, float(v)) for v in r]).reshape(z.shape)
    return lam * 0.5 * b


def weights(f, reg: O.Reg):
    """(Wr, Wd, W0): Wr[n, m] for the edge (n, m) -> (n, m + 1), shape
    (N, N - 1); Wd[n, m] for (n, m) -> (n + 1, m), shape (N - 1, N); W0[n, m]
    for the pixel.  Zero where the lambda of the term is zero."""
    f = np.asarray(f, np.complex128)
    N = f.shape[0]
    if reg.lambda1 != 0.0:
        Wr = _w(reg.kind, reg.alpha1, reg.lambda1, f[:, 1:] - f[:, :-1])
        Wd = _w(reg.kind, reg.alpha1, reg.lambda1, f[1:, :] - f[:-1, :])
    else:
        Wr, Wd = np.zeros((N, N - 1)), np.zeros((N - 1, N))
    W0 = _w(reg.kind, reg.alpha0, reg.lambda0, f) if reg.lambda0 != 0.0 else np.zeros((N, N))
    return Wr, Wd, W0


def penalty_normal(x, W):
    """sum_e W_e delta_e^H delta_e x: an edge p -> q with z = x_q - x_p adds
    W_e z at q and -W_e z at p; a pixel adds W0 x_p."""
    Wr, Wd, W0 = W
    x = np.asarray(x, np.complex128)
    out = W0 * x
    zr = Wr * (x[:, 1:] - x[:, :-1])
    out[:, 1:] += zr
    out[:, :-1] -= zr
    zd = Wd * (x[1:, :] - x[:-1, :])
    out[1:, :] += zd
    out[:-1, :] -= zd
    return out


def normal_apply(kx, ky, x, W):
    """A x = H^H H x + sum_e W_e delta_e^H delta_e x."""
    N = x.shape[0]
    return O.adjoint(kx, ky, O.forward(kx, ky, x), N) + penalty_normal(x, W)


def surrogate(kx, ky, s, f, fk, reg: O.Reg):
    """K(f, W(f^k)) + sum_e psi(W_e): the half-quadratic majorant of J at f^k,
    ||s - H f||^2 + sum_e [lambda_e phi(r_e^k) + lambda_e W'_e (|z_e(f)|^2 -
    (r_e^k)^2)] with W = lambda W'."""
    f = np.asarray(f, np.complex128)
    fk = np.asarray(fk, np.complex128)
    data = float(np.sum(np.abs(s - O.forward(kx, ky, f)) ** 2))
    W = weights(fk, reg)
    terms = 0.0
    parts = [(reg.lambda1, reg.alpha1, W[0], lambda x: x[:, 1:] - x[:, :-1]),
             (reg.lambda1, reg.alpha1, W[1], lambda x: x[1:, :] - x[:-1, :]),
             (reg.lambda0, reg.alpha0, W[2], lambda x: x)]
    for lam, alpha, w, z in parts:
        if lam == 0.0:
            continue
        rk = np.abs(z(fk))
        phik = np.array([O.phi(reg.kind, alpha, float(v)) for v in rk.ravel()]).reshape(rk.shape)
        terms += float(np.sum(lam * phik + w * (np.abs(z(f)) ** 2 - rk ** 2)))
    return data + terms


def solve(kx, ky, s, reg: O.Reg, x0, outer, inner):
    """outer half-quadratic steps of inner linear CG steps each from x0.
    Returns (x, J_hist[outer + 1]) with J_hist[k] = J(f^k)."""
    kx = np.ascontiguousarray(kx, np.float64)
    ky = np.ascontiguousarray(ky, np.float64)
    s = np.asarray(s, np.complex128)
    f = np.array(x0, np.complex128)
    N = f.shape[0]
    D = O.adjoint(kx, ky, s, N)
    Js = [O.objective(kx, ky, s, f, reg)]
    for _ in range(outer):
        W = weights(f, reg)
        r = D - normal_apply(kx, ky, f, W)
        p = r.copy()
        rho = _redot(r, r)
        for _ in range(inner):
            q = normal_apply(kx, ky, p, W)
            pq = _redot(p, q)
            alpha = rho / pq if pq > 0.0 else 0.0
            f = f + alpha * p
            r = r - alpha * q
            rho_new = _redot(r, r)
            beta = rho_new / rho if rho > 0.0 else 0.0
            p = r + beta * p
            rho = rho_new
        Js.append(O.objective(kx, ky, s, f, reg))
    return f, np.array(Js)
