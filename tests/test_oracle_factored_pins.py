"""Pins of oracle/factored.py (the forward, adjoint and G sums taken as
matrix products of phase matrices) against the direct double-loop sums of the
C oracle and against the complete Cartesian grid, where H is a scaled inverse
DFT (section 3.1, Eq. InvCart)."""
import numpy as np
import pytest

from oracle import factored as F
from oracle import oracle as O
from paper_0908_3252_gb300 import synth


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


@pytest.mark.parametrize("N,L", [(2, 1), (8, 50), (37, 999), (64, 3000)])
def test_equals_the_direct_sums(N, L):
    """Same sums, another summation order: FP64 rounding apart (a transposed
    phase matrix, a dropped conjugate or a wrong scale fails by O(1))."""
    g = synth.rng(N + L)
    kx, ky = synth.uniform_k(L, g)
    f = synth.complex_normal((N, N), g)
    s = synth.complex_normal(L, g)
    assert rel(F.forward(kx, ky, f), O.forward(kx, ky, f)) < 1e-12
    assert rel(F.adjoint(kx, ky, s, N), O.adjoint(kx, ky, s, N)) < 1e-12
    assert rel(F.gram(kx, ky, N), O.gram(kx, ky, N)) < 1e-12


def test_cartesian_grid():
    """Complete grid: H f = N ifft2(f) (numpy's FFT) and G = delta."""
    N = 12
    kx, ky = synth.cartesian(N)
    f = synth.complex_normal((N, N), synth.rng(2))
    Fq = N * np.fft.ifft2(f)
    jx = np.rint(kx * N).astype(int) % N
    jy = np.rint(ky * N).astype(int) % N
    assert rel(F.forward(kx, ky, f), Fq[jy, jx]) < 1e-12
    assert rel(F.adjoint(kx, ky, F.forward(kx, ky, f), N), f) < 1e-12
    G = F.gram(kx, ky, N)
    assert abs(G[N - 1, N - 1] - 1.0) < 1e-12
    G[N - 1, N - 1] = 0.0
    assert np.max(np.abs(G)) < 1e-12


def test_sampled_entries_at_a_larger_size():
    """N = 128, L = 16384 spiral: sampled lags of G and pixels of D against
    the C oracle's single-entry sums."""
    N = 128
    kx, ky = synth.spiral(N, 8, 2048, "archimedean")
    g = synth.rng(5)
    s = synth.complex_normal(kx.shape[0], g)
    G = F.gram(kx, ky, N)
    u = g.integers(-(N - 1), N, 24).astype(np.int32)
    v = g.integers(-(N - 1), N, 24).astype(np.int32)
    assert rel(G[v + N - 1, u + N - 1], O.gram_at(kx, ky, N, u, v)) < 1e-12
    D = F.adjoint(kx, ky, s, N)
    n = g.integers(0, N, 24).astype(np.int32)
    m = g.integers(0, N, 24).astype(np.int32)
    assert rel(D[n, m], O.adjoint_at(kx, ky, s, N, n, m)) < 1e-12
