"""spirec_toeplitz_noalloc: the Toeplitz apply for callers that cannot
allocate device memory (a fixed memory budget, no footprint growth after
start-up).  Its scratch is a file-scope device array, so it needs no plan and
no cudaMalloc.  Checked through the C ABI against spirec_toeplitz_dev (the
plan-based entry point) on two calls in a row, with different inputs, so a
call that left stale state in the shared array would show; against the FP64
oracle's H^H (H x) (Appendix B); at its size limit (N = 512, M = 1024,
sampled pixels of a sparse x against the oracle's G sums); and with the grid
size changing between calls (M = 64, then 1024, then 64 again).

This file is named to be collected last: if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0908_3252_gb300 import synth
from tests.helpers import c64, empty_c64, from_dev, rel, to_dev, workload_c1, workload_ragged

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the FP32 tolerance of the other parity tests


@pytest.fixture(scope="module")
def sp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0908_3252_gb300 import build, spirec
    build.build()
    spirec.load()
    return spirec


def _spectrum(sp, p):
    import torch
    spec = torch.zeros((p.M, p.M), dtype=torch.float32, device="cuda:0")
    sp.spirec_kernel_spectrum_dev(p.h, spec)
    return spec


@pytest.mark.parametrize("wname,M", [("c1", 0), ("ragged", 75)])
def test_noalloc_matches_plan_toeplitz_and_oracle(sp, wname, M):
    import torch
    w = workload_c1() if wname == "c1" else workload_ragged()
    N = w["N"]
    stream = torch.cuda.current_stream().cuda_stream
    with sp.Plan(N, w["kx"].shape[0], M, 0, stream, w["kx"], w["ky"]) as p:
        spec = _spectrum(sp, p)
        g = synth.rng(31)
        for call in range(2):
            xh = c64(synth.complex_normal((N, N), g))
            x = to_dev(xh)
            want = empty_c64((N, N))
            sp.spirec_toeplitz_dev(p.h, x, want)
            got = empty_c64((N, N))
            sp.spirec_toeplitz_noalloc(x, spec, got, N, p.M, stream)
            got = from_dev(got)
            assert rel(got, from_dev(want)) < TOL, f"call {call}"
            oracle = O.adjoint(w["kx"], w["ky"], O.forward(w["kx"], w["ky"], xh), N)
            assert rel(got, oracle) < TOL, f"call {call}"


def _sparse_case(N, seed):
    """x with three nonzero pixels, and sampled pixels of T x from the
    oracle's G sums: (T x)[n][m] = sum_j x_j conj(G_{m - m_j, n - n_j})."""
    g = synth.rng(seed)
    pts = [(0, 0), (N - 1, N - 1), (N // 3, 17)]
    vals = c64(synth.complex_normal(3, g))
    x = np.zeros((N, N), np.complex64)
    for (a, b), val in zip(pts, vals):
        x[a, b] = val
    n = np.concatenate([[0, N - 1, N // 3], g.integers(0, N, 29)])
    m = np.concatenate([[0, N - 1, 17], g.integers(0, N, 29)])
    return x, pts, vals, n, m


def test_noalloc_at_its_size_limit_and_after_a_grid_change(sp):
    """N = 512, M = 1024 (the array's limit: rows, transposed spectrum and
    twiddles fill it), between two calls at M = 64 on another problem."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    small = workload_c1()
    Ns = small["N"]
    N = 512
    kx, ky = synth.spiral(N, 8, 2048, "archimedean")
    with sp.Plan(Ns, small["kx"].shape[0], 0, 0, stream, small["kx"], small["ky"]) as ps, \
            sp.Plan(N, kx.shape[0], 1024, 0, stream, kx, ky) as pl:
        spec_s, spec_l = _spectrum(sp, ps), _spectrum(sp, pl)
        xs = to_dev(c64(synth.complex_normal((Ns, Ns), synth.rng(41))))
        want_s = empty_c64((Ns, Ns))
        sp.spirec_toeplitz_dev(ps.h, xs, want_s)
        want_s = from_dev(want_s)
        x, pts, vals, n, m = _sparse_case(N, 42)
        xd = to_dev(x)
        want_l = empty_c64((N, N))
        sp.spirec_toeplitz_dev(pl.h, xd, want_l)
        want_l = from_dev(want_l)
        got_l = None
        for label in ("before", "after"):
            got_s = empty_c64((Ns, Ns))
            sp.spirec_toeplitz_noalloc(xs, spec_s, got_s, Ns, ps.M, stream)
            assert rel(from_dev(got_s), want_s) < TOL, label
            if label == "before":
                out_l = empty_c64((N, N))
                sp.spirec_toeplitz_noalloc(xd, spec_l, out_l, N, 1024, stream)
                got_l = from_dev(out_l)  # host copy (N x N)
                assert rel(got_l, want_l) < TOL
    assert got_l.shape == (N, N) and isinstance(got_l, np.ndarray)
    u = np.array([[mm - b for (a, b) in pts] for mm in m]).ravel().astype(np.int32)
    v = np.array([[nn - a for (a, b) in pts] for nn in n]).ravel().astype(np.int32)
    Gs = O.gram_at(kx, ky, N, u, v).reshape(len(n), 3)
    oracle = (np.conj(Gs) * vals[None, :]).sum(axis=1)
    assert rel(got_l[n, m], oracle) < TOL


def test_noalloc_rejects_sizes_beyond_its_array(sp):
    import torch
    N, M = 600, 1200
    x = torch.zeros((8,), dtype=torch.complex64, device="cuda:0")
    spec = torch.zeros((8,), dtype=torch.float32, device="cuda:0")
    with pytest.raises(sp.SpirecError) as e:
        sp.spirec_toeplitz_noalloc(x, spec, x, N, M)
    assert e.value.code == sp.SPIREC_EINVAL
    assert "512" in str(e.value)
    with pytest.raises(sp.SpirecError) as e:
        sp.spirec_toeplitz_noalloc(x, spec, x, 32, 40)  # M < 2N - 1
    assert e.value.code == sp.SPIREC_EINVAL
    with pytest.raises(sp.SpirecError) as e:
        sp.spirec_toeplitz_noalloc(x, spec, x, 512, 1030)  # M beyond the array
    assert e.value.code == sp.SPIREC_EINVAL
