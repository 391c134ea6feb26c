"""The paper's method on the CPU, in FP64 (test infrastructure and a CPU
baseline; shares no code with the CUDA path and is never called by it).

The criterion in its rewritten form (section 3.4, Eq. NewCritLS):
    J(f) = ||s||^2 - 2 Re<f, D> + Re<f, T f> + R(f),   D = H^H s,
with the normal operator T = H^H H applied as the Toeplitz convolution of
Appendix B through zero-padded FFTs (scipy.fft on the host cores), and the
same minimiser as oracle.solve: PR+ CG with a descent restart and three
majorize-minimize line-search steps on h(t) = J(f + t d).  G and D come from
the oracle's direct sums, or, for full-size problems (problem_fp64), from the
same sums taken as matrix products (oracle/factored.py).  The pin in
tests/test_oracle_pins.py checks this solve against oracle.solve (direct
NUDFTs) to FP64 rounding, which checks the rewriting itself.
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft as sfft

from oracle import oracle as O

WORKERS = os.cpu_count() or 1


def kernel_spectrum(G_full: np.ndarray, N: int, M: int) -> np.ndarray:
    """FFT2 of the M x M circulant c[v mod M][u mod M] = conj G_{u,v}
    (|u|, |v| <= N-1; zero elsewhere).  G_full is indexed [v+N-1, u+N-1]."""
    lag = np.arange(-(N - 1), N)
    c = np.zeros((M, M), np.complex128)
    c[np.ix_(lag % M, lag % M)] = np.conj(G_full)
    return sfft.fft2(c, workers=WORKERS)


def toeplitz_apply(C_hat: np.ndarray, x: np.ndarray) -> np.ndarray:
    """(T x)[n][m] = sum x[n'][m'] conj G_{m-m', n-n'} = crop_N(IFFT2(C_hat FFT2(pad_M x)))."""
    N, M = x.shape[0], C_hat.shape[0]
    xp = np.zeros((M, M), np.complex128)
    xp[:N, :N] = x
    return sfft.ifft2(C_hat * sfft.fft2(xp, workers=WORKERS), workers=WORKERS)[:N, :N]


def problem_fp64(kx, ky, s, N: int, M: int):
    """The rewritten problem in FP64 for any size: (C_hat, D, ||s||^2) with
    G (Eq. AnnMatG) and D (Eq. AnnMatGD) from oracle/factored.py."""
    from oracle import factored as F
    s = np.asarray(s, np.complex128)
    C_hat = kernel_spectrum(F.gram(kx, ky, N), N, M)
    return C_hat, F.adjoint(kx, ky, s, N), float(np.sum(np.abs(s) ** 2))


def _weight(kind: int, alpha: float, r: np.ndarray) -> np.ndarray:
    """b(r) = phi'(r) / r (as oracle.phi_weight, vectorised)."""
    if kind == O.PHI_HUBER:
        return np.where(r <= alpha, 2.0, 2.0 * alpha / np.maximum(r, 1e-300))
    if kind == O.PHI_HYPERBOLIC:
        return 2.0 * alpha / np.sqrt(alpha * alpha + r * r)
    return np.full_like(r, 2.0)


def _line_terms(f: np.ndarray, d: np.ndarray, t: float, reg: O.Reg) -> tuple[float, float]:
    """Penalty parts of h'(t) and of the majorant's curvature: sums over the
    down and right differences (free boundary) and the pixels of
    lambda b(|z + t w|) Re(conj(z + t w) w) and lambda b(|z + t w|) |w|^2."""
    num = den = 0.0
    for z, w, lam, alpha in ((f[1:, :] - f[:-1, :], d[1:, :] - d[:-1, :], reg.lambda1, reg.alpha1),
                             (f[:, 1:] - f[:, :-1], d[:, 1:] - d[:, :-1], reg.lambda1, reg.alpha1),
                             (f, d, reg.lambda0, reg.alpha0)):
        if lam == 0.0:
            continue
        x = z + t * w
        b = lam * _weight(reg.kind, alpha, np.abs(x))
        num += float(np.sum(b * (x.real * w.real + x.imag * w.imag)))
        den += float(np.sum(b * (w.real * w.real + w.imag * w.imag)))
    return num, den


def _redot(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.sum(a.real * b.real + a.imag * b.imag))


def solve(C_hat: np.ndarray, D: np.ndarray, ss: float, reg: O.Reg, x0: np.ndarray, iters: int):
    """The minimiser of oracle.solve on the rewritten criterion.  C_hat from
    kernel_spectrum, D = H^H s, ss = ||s||^2.  Returns (x, J_hist)."""
    f = np.array(x0, np.complex128)
    Tf = toeplitz_apply(C_hat, f)

    def grad_and_J(f, Tf):
        g_ls = 2.0 * (Tf - D)
        g = g_ls + O.penalty_grad(f, reg)
        J = ss - 2.0 * _redot(f, D) + _redot(f, Tf) + O.penalty(f, reg)
        return g, g_ls, J

    g, g_ls, J = grad_and_J(f, Tf)
    Js = [J]
    d = -g
    for _ in range(iters):
        Td = toeplitz_apply(C_hat, d)
        q2 = _redot(d, Td)
        q1 = _redot(d, g_ls)
        t = 0.0
        for _ in range(3):
            num, den = _line_terms(f, d, t, reg)
            num += q1 + 2.0 * q2 * t
            den += 2.0 * q2
            if den > 0.0:
                t -= num / den
        f = f + t * d
        Tf = Tf + t * Td
        gn, g_ls, J = grad_and_J(f, Tf)
        Js.append(J)
        gg_old = _redot(g, g)
        beta = max(0.0, _redot(gn, gn - g) / gg_old) if gg_old > 0.0 else 0.0
        d = -gn + beta * d
        if _redot(gn, d) >= 0.0:
            d = -gn
        g = gn
    return f, np.array(Js)
