"""FP64 forward, adjoint and G for full-size problems: each sum over the
samples taken by one matrix product of phase matrices.

TEST INFRASTRUCTURE ONLY.  Nothing in the product library imports or calls
this module; only the tests and the benchmark's CPU leg do.  It shares no code
with the CUDA path.  It is pinned to the direct double-loop sums of
spirec_oracle.c (tests/test_oracle_factored_pins.py), which it reproduces to
FP64 rounding; it exists because those sums take minutes at 512^2 with
L = 131072, where these take seconds.

Every term of the three sums has the phase exp(+-i 2 pi (kx_l m + ky_l n)),
the product of exp(+-i 2 pi kx_l m) and exp(+-i 2 pi ky_l n) (the exponential
of a sum).  Each factor is formed with the direct oracle's exact range
reduction (theta - round(theta), cycles, before the trig call).  With the
phase matrices
    Ex[l, m] = exp(+i 2 pi kx_l m),   Ey[l, n] = exp(+i 2 pi ky_l n)
the sums of section 2 and Appendix A read
    (H f)_l  = (1/N)   sum_n Ey[l, n] sum_m Ex[l, m] f[n][m]          (Eq. ModDirect)
    D[n][m]  = (1/N)   sum_l conj(Ey[l, n]) s_l conj(Ex[l, m])         (Eq. AnnMatGD)
    G_{u,v}  = (1/N^2) sum_l Ex[l, u] Ey[l, v],  u, v in [1-N, N-1]    (Eq. AnnMatG)
and each sum over l (or over m) is one numpy matrix product.  Images are
(N, N) arrays [n, m] with n the row (ky) and m the column (kx); G is returned
as a (2N-1, 2N-1) array indexed [v+N-1, u+N-1], as oracle.gram does.
"""
from __future__ import annotations

import numpy as np


def phases(k: np.ndarray, j: np.ndarray, sign: float = 1.0) -> np.ndarray:
    """E[l, i] = exp(sign i 2 pi k_l j_i), the phase reduced to [-0.5, 0.5]
    cycles before the trig call (L x len(j), complex128)."""
    theta = np.multiply.outer(np.asarray(k, np.float64), np.asarray(j, np.float64))
    theta -= np.rint(theta)
    a = 2.0 * np.pi * theta
    return np.cos(a) + 1j * (sign * np.sin(a))


def forward(kx, ky, f):
    """y = H f (Eq. ModDirect)."""
    f = np.asarray(f, np.complex128)
    N = f.shape[0]
    idx = np.arange(N)
    Ex = phases(kx, idx)
    Ey = phases(ky, idx)
    Z = Ex @ f.T  # Z[l, n] = sum_m Ex[l, m] f[n][m]
    return np.sum(Ey * Z, axis=1) / N


def adjoint(kx, ky, r, N):
    """x = H^H r; with r = s this is D (Eq. AnnMatGD)."""
    r = np.asarray(r, np.complex128)
    idx = np.arange(N)
    Ex = phases(kx, idx, -1.0)
    Ey = phases(ky, idx, -1.0)
    return (Ey.T @ (r[:, None] * Ex)) / N


def gram(kx, ky, N):
    """Every lag of G (Eq. AnnMatG), indexed [v+N-1, u+N-1]."""
    lag = np.arange(-(N - 1), N)
    Ex = phases(kx, lag)
    Ey = phases(ky, lag)
    return (Ey.T @ Ex) / (float(N) * N)
