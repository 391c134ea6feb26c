"""Parity at the benchmark's full size (N = 512, L = 32 x 4096 = 131072,
M = 1024), in the benchmark's launch configuration, on outputs the FP64 oracle
can compute one at a time: sampled lags of G, sampled pixels of D, sampled
samples of H x, and T x for a sparse x at sampled pixels (T x is then a short
sum of G values).  Plus properties that hold at any size for the solve.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0908_3252_gb300 import synth
from tests.helpers import c64, empty_c64, from_dev, rel, to_dev

pytestmark = pytest.mark.gpu

N, I, S, M = 512, 32, 4096, 1024
TOL = {0: 1e-5, 1: 1e-3, 2: 1e-3}
PRECISIONS = [0, 1, 2]


@pytest.fixture(scope="module")
def sp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0908_3252_gb300 import build, spirec
    build.build()
    spirec.load()
    return spirec


@pytest.fixture(scope="module")
def traj():
    kx, ky = synth.spiral(N, I, S, "archimedean")
    return kx, ky


@pytest.fixture(scope="module", params=PRECISIONS)
def plan(sp, traj, request):
    import torch
    kx, ky = traj
    p = sp.Plan(N, kx.shape[0], M, request.param, torch.cuda.current_stream().cuda_stream, kx, ky)
    yield request.param, p
    p.close()


def test_gram_sampled(sp, traj, plan):
    prec, p = plan
    kx, ky = traj
    G = empty_c64((N, 2 * N - 1))
    sp.spirec_gram_dev(p.h, G)
    G = from_dev(G)
    g = synth.rng(101)
    u = np.concatenate([[0, 0, N - 1, 1], g.integers(0, N, 60)]).astype(np.int32)
    v = np.concatenate([[0, -(N - 1), N - 1, -1], g.integers(-(N - 1), N, 60)]).astype(np.int32)
    want = O.gram_at(kx, ky, N, u, v)
    got = G[u, v + N - 1]
    print(f"precision {prec}: sampled G {rel(got, want):.2e} from the FP64 sums")
    assert rel(got, want) < TOL[prec]


def test_adjoint_sampled(sp, traj, plan):
    prec, p = plan
    kx, ky = traj
    g = synth.rng(102)
    s = c64(synth.complex_normal(kx.shape[0], g))
    sp.spirec_set_data(p.h, s)
    D = empty_c64((N, N))
    sp.spirec_data_adjoint_dev(p.h, D)
    D = from_dev(D)
    n = g.integers(0, N, 48).astype(np.int32)
    m = g.integers(0, N, 48).astype(np.int32)
    want = O.adjoint_at(kx, ky, s, N, n, m)
    print(f"precision {prec}: sampled D {rel(D[n, m], want):.2e} from the FP64 sums")
    assert rel(D[n, m], want) < TOL[prec]


def test_forward_sampled(sp, traj, plan):
    prec, p = plan
    kx, ky = traj
    g = synth.rng(103)
    x = c64(synth.complex_normal((N, N), g))
    y = empty_c64((kx.shape[0],))
    sp.spirec_forward_dev(p.h, to_dev(x), y)
    y = from_dev(y)
    idx = g.integers(0, kx.shape[0], 24)
    want = O.forward(kx[idx], ky[idx], x)
    assert rel(y[idx], want) < TOL[prec]


def test_toeplitz_sparse_sampled(sp, traj, plan):
    """x with 3 nonzero pixels: (T x)[n][m] = sum_j x_j conj(G_{m-m_j, n-n_j})."""
    prec, p = plan
    kx, ky = traj
    g = synth.rng(104)
    pts = [(0, 0), (N - 1, N - 1), (200, 17)]
    vals = c64(synth.complex_normal(3, g))
    x = np.zeros((N, N), np.complex64)
    for (a, b), val in zip(pts, vals):
        x[a, b] = val
    Tx = empty_c64((N, N))
    sp.spirec_toeplitz_dev(p.h, to_dev(x), Tx)
    Tx = from_dev(Tx)
    n = np.concatenate([[0, N - 1, 200], g.integers(0, N, 29)])
    m = np.concatenate([[0, N - 1, 17], g.integers(0, N, 29)])
    u = np.array([[mm - b for (a, b) in pts] for mm in m]).ravel().astype(np.int32)
    v = np.array([[nn - a for (a, b) in pts] for nn in n]).ravel().astype(np.int32)
    Gs = O.gram_at(kx, ky, N, u, v).reshape(len(n), 3)
    want = (np.conj(Gs) * vals[None, :]).sum(axis=1)
    assert rel(Tx[n, m], want) < TOL[prec]


def test_solve_properties(sp, traj, plan):
    """50 iterations of the benchmark workload: J finite and non-increasing,
    and the final J equals J recomputed from the returned iterate."""
    prec, p = plan
    kx, ky = traj
    g = synth.rng(105)
    f_true = synth.phantom(N, "edges_texture", g)
    x = to_dev(c64(f_true))
    y = empty_c64((kx.shape[0],))
    sp.spirec_forward_dev(p.h, x, y)
    s = synth.add_noise(from_dev(y).astype(np.complex128), 30.0, g).astype(np.complex64)
    sp.spirec_set_data(p.h, s)
    sp.spirec_set_reg(p.h, 0.05, 0.05, 0.0, 0.05, 0)
    xr, J = sp.spirec_solve(p.h, None, 50, N)
    assert np.all(np.isfinite(J))
    assert np.all(np.diff(J) <= 1e-6 * J[0])
    assert J[-1] < 0.05 * J[0]
    gd = empty_c64((N, N))
    J2 = sp.spirec_objective_grad_dev(p.h, to_dev(xr), gd)
    # both are differences of terms of size ||s||^2 = J[0] (x0 = 0)
    assert abs(J2 - J[-1]) < 1e-5 * J[0]
