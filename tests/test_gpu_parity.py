"""GPU parity: every operator of the CUDA path against the FP64 oracle, called
through the C ABI (libspirec.so).

Tolerances (relative L2 against the FP64 oracle, same inputs on both sides):
  FP32 path            1e-5   (the FP32 tolerance of the reconstruction target)
  FP16x3 / BF16x3 path 1e-3   (mixed-precision contraction target)
applied to every result with a plain definition: G, D, H x, T x, the kernel
spectrum, the J history of a solve, and the iterate after the first three
iterations.  Two quantities are differences of much larger terms in the
rewritten criterion (section 3.4), so the bar is stated against those terms:
  grad J = 2 (T x - D) + grad R   -> ||err|| <= tol * (2||T x|| + 2||D|| + ||grad R||)
  J = ||s||^2 - 2 Re<x,D> + Re<x,T x> + R -> |err| <= tol * (sum of |terms|)
The iterate after 30-50 nonlinear CG iterations is held at the target or at
3 x the distance the FP32 rounding model of the same minimiser shows from the
oracle on the same problem, whichever is larger (tests.helpers.iter_tol,
oracle/fp32_model.py): an FP32 implementation of the method cannot land
closer than that model on these problems.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0908_3252_gb300 import synth
from tests.helpers import c64, empty_c64, from_dev, iter_tol, rel, to_dev, workload_c1, workload_ragged

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-3, 2: 1e-3}
PRECISIONS = [0, 1, 2]


def _terms(w, x, reg):
    """Magnitudes of the terms the rewritten J and grad J combine (oracle)."""
    kx, ky, s, N = w["kx"], w["ky"], w["s"], w["N"]
    D = O.adjoint(kx, ky, s, N)
    Tx = O.adjoint(kx, ky, O.forward(kx, ky, x), N)
    gR = O.penalty_grad(x, reg)
    J_terms = (np.sum(np.abs(s) ** 2) + 2 * abs(np.vdot(x, D)) + abs(np.vdot(x, Tx))
               + O.penalty(x, reg))
    g_terms = 2 * np.linalg.norm(Tx) + 2 * np.linalg.norm(D) + np.linalg.norm(gR)
    return J_terms, g_terms


@pytest.fixture(scope="module")
def sp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0908_3252_gb300 import build, spirec
    build.build()
    spirec.load()
    return spirec


def _plan(sp, w, prec, M=0):
    import torch
    L = w["kx"].shape[0]
    p = sp.Plan(w["N"], L, M, prec, torch.cuda.current_stream().cuda_stream, w["kx"], w["ky"])
    return p


def _half(Gfull, N):
    # oracle G indexed [v+N-1, u+N-1] -> plan layout [u][v+N-1] for u >= 0
    return Gfull[:, N - 1:].T


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("wname", ["c1", "ragged"])
def test_gram(sp, prec, wname):
    w = workload_c1() if wname == "c1" else workload_ragged()
    N = w["N"]
    with _plan(sp, w, prec) as p:
        G = empty_c64((N, 2 * N - 1))
        sp.spirec_gram_dev(p.h, G)
        got = from_dev(G)
    want = _half(O.gram(w["kx"], w["ky"], N), N)
    assert rel(got, want) < TOL[prec]


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("wname", ["c1", "ragged"])
def test_adjoint_D(sp, prec, wname):
    w = workload_c1() if wname == "c1" else workload_ragged()
    N = w["N"]
    with _plan(sp, w, prec) as p:
        sp.spirec_set_data(p.h, w["s"])
        D = empty_c64((N, N))
        sp.spirec_data_adjoint_dev(p.h, D)
        got = from_dev(D)
    want = O.adjoint(w["kx"], w["ky"], w["s"], N)
    assert rel(got, want) < TOL[prec]


@pytest.mark.parametrize("wname", ["c1", "ragged"])
@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("scale", [1.0, 3e5, 1e-6])
def test_forward(sp, wname, prec, scale):
    """H x (Eq. ModDirect); the mixed paths run it as a tensor-core
    contraction on an FP16/BF16 split of x, scaled by a power of two into
    range (images of 3e5 would overflow FP16 unscaled, 1e-6 would underflow)."""
    w = workload_c1() if wname == "c1" else workload_ragged()
    x = c64(scale * w["f_true"])
    with _plan(sp, w, prec) as p:
        xd = to_dev(x)
        y = empty_c64((w["kx"].shape[0],))
        sp.spirec_forward_dev(p.h, xd, y)
        got = from_dev(y)
    assert rel(got, O.forward(w["kx"], w["ky"], x)) < TOL[prec]


@pytest.mark.parametrize("wname", ["c1", "ragged"])
def test_toeplitz_equals_normal_operator(sp, wname):
    """T x by the zero-padded FFT equals the oracle's H^H (H x) (Appendix B)."""
    w = workload_c1() if wname == "c1" else workload_ragged()
    N = w["N"]
    g = synth.rng(5)
    x = c64(synth.complex_normal((N, N), g))
    with _plan(sp, w, 0) as p:
        Tx = empty_c64((N, N))
        sp.spirec_toeplitz_dev(p.h, to_dev(x), Tx)
        got = from_dev(Tx)
    want = O.adjoint(w["kx"], w["ky"], O.forward(w["kx"], w["ky"], x), N)
    assert rel(got, want) < 1e-5


@pytest.mark.parametrize("N,M", [(259, 2048), (601, 4096)])
def test_toeplitz_split_passes(sp, N, M):
    """T x at M = 2048 and 4096, where the row and column passes split every
    transform into 2 or 4 warp-sized 1024-point DFTs, on images whose row
    count leaves a partial last row group (4 rows a group at M = 2048, 2 at
    4096), against the oracle's H^H (H x)."""
    g = synth.rng(N)
    kx, ky = synth.spiral(N, 2, 300, "variable")
    w = dict(N=N, kx=kx, ky=ky)
    x = c64(synth.complex_normal((N, N), g))
    with _plan(sp, w, 0, M=M) as p:
        assert p.M == M
        Tx = empty_c64((N, N))
        sp.spirec_toeplitz_dev(p.h, to_dev(x), Tx)
        got = from_dev(Tx)
    want = O.adjoint(kx, ky, O.forward(kx, ky, x), N)
    assert rel(got, want) < 1e-5


def test_spectrum_is_the_embedded_gram(sp):
    """Chat = Re FFT2(c) / M^2 with c[v mod M][u mod M] = conj G_{u,v}."""
    w = workload_ragged(N=20, I=2, S=150)
    N = w["N"]
    with _plan(sp, w, 0) as p:
        M = p.M
        import torch
        C = torch.zeros((M, M), dtype=torch.float32, device="cuda:0")
        sp.spirec_kernel_spectrum_dev(p.h, C)
        got = from_dev(C)
    G = O.gram(w["kx"], w["ky"], N)
    c = np.zeros((M, M), np.complex128)
    for v in range(-(N - 1), N):
        for u in range(-(N - 1), N):
            c[v % M, u % M] = np.conj(G[v + N - 1, u + N - 1])
    spec = np.fft.fft2(c) / M ** 2
    assert np.max(np.abs(spec.imag)) < 1e-12 * np.max(np.abs(spec.real)) + 1e-15
    assert rel(got, spec.real) < 1e-5


@pytest.mark.parametrize("kind", [O.PHI_HUBER, O.PHI_HYPERBOLIC, O.PHI_QUADRATIC])
def test_objective_and_gradient(sp, kind):
    w = workload_ragged(kind=kind)
    N, reg = w["N"], w["reg"]
    g = synth.rng(17)
    x = c64(w["f_true"] + 0.1 * synth.complex_normal((N, N), g))
    with _plan(sp, w, 0) as p:
        sp.spirec_set_data(p.h, w["s"])
        sp.spirec_set_reg(p.h, reg.lambda1, reg.alpha1, reg.lambda0, reg.alpha0, reg.kind)
        gd = empty_c64((N, N))
        J = sp.spirec_objective_grad_dev(p.h, to_dev(x), gd)
        got = from_dev(gd)
    J_terms, g_terms = _terms(w, x, reg)
    go = O.gradient(w["kx"], w["ky"], w["s"], x, reg)
    assert np.linalg.norm(got - go) < 1e-5 * g_terms
    Jo = O.objective(w["kx"], w["ky"], w["s"], x, reg)
    assert abs(J - Jo) < 1e-5 * J_terms


def _solve_both(sp, w, prec, x0=None):
    N, reg, iters = w["N"], w["reg"], w["iters"]
    with _plan(sp, w, prec) as p:
        sp.spirec_set_data(p.h, w["s"])
        sp.spirec_set_reg(p.h, reg.lambda1, reg.alpha1, reg.lambda0, reg.alpha0, reg.kind)
        x, J = sp.spirec_solve(p.h, x0, iters, N)
    xo, Jo, _ = O.solve(w["kx"], w["ky"], w["s"], reg,
                        np.zeros((N, N)) if x0 is None else c64(x0), iters)
    return x, J, xo, Jo


@pytest.mark.parametrize("prec", PRECISIONS)
def test_solve_c1(sp, prec):
    """32x32 workload, 50 iterations: J history and iterates against the oracle."""
    w = workload_c1()
    x, J, xo, Jo = _solve_both(sp, w, prec)
    assert np.all(np.isfinite(J))
    assert np.all(np.diff(J) <= 1e-6 * J[0]), "J must not increase"
    assert rel(J, Jo) < TOL[prec]
    assert rel(x, xo) < iter_tol(w, prec), (rel(x, xo), iter_tol(w, prec))
    w3 = dict(w, iters=3)
    x3, _, xo3, _ = _solve_both(sp, w3, prec)
    assert rel(x3, xo3) < TOL[prec]


def test_solve_ragged_with_x0(sp):
    w = workload_ragged()
    g = synth.rng(3)
    x0 = (0.5 * w["f_true"] + 0.05 * synth.complex_normal(w["f_true"].shape, g)).astype(np.complex64)
    x, J, xo, Jo = _solve_both(sp, w, 0, x0)
    assert np.all(np.diff(J) <= 1e-6 * J[0])
    assert rel(J, Jo) < 1e-5
    assert rel(x, xo) < iter_tol(w, 0, x0), (rel(x, xo), iter_tol(w, 0, x0))
    x3, _, xo3, _ = _solve_both(sp, dict(w, iters=3), 0, x0)
    assert rel(x3, xo3) < 1e-5


def test_solve_zero_iterations_returns_x0(sp):
    w = workload_ragged(N=16, I=2, S=100)
    w["iters"] = 0
    x0 = w["f_true"].astype(np.complex64)
    x, J, xo, Jo = _solve_both(sp, w, 0, x0)
    assert np.array_equal(x, x0)
    J_terms, _ = _terms(w, c64(x0), w["reg"])
    assert abs(J[0] - Jo[0]) < 1e-5 * J_terms


def test_smallest_sizes(sp):
    """N = 2, L = 1: every tile is a ragged tail."""
    N = 2
    kx, ky = np.array([0.21]), np.array([-0.37])
    w = dict(N=N, kx=kx, ky=ky, s=c64(np.array([0.3 - 0.2j])),
             reg=O.Reg(0.1, 0.05, 0.01, 0.05, O.PHI_HUBER), iters=4,
             f_true=np.zeros((N, N)))
    x, J, xo, Jo = _solve_both(sp, w, 0)
    assert rel(x, xo) < 1e-5
    assert rel(J, Jo) < 1e-5


def test_cartesian_grid_inverts_exactly(sp):
    """Complete Cartesian grid, lambda = 0: one iteration returns H^H s = f."""
    N = 16
    kx, ky = synth.cartesian(N)
    f = synth.phantom(N, "ellipses_phase", synth.rng(8))
    s = c64(O.forward(kx, ky, f))
    w = dict(N=N, kx=kx, ky=ky, s=s, reg=O.Reg(0.0, 1.0, 0.0, 1.0, O.PHI_HUBER), iters=1, f_true=f)
    x, J, xo, Jo = _solve_both(sp, w, 0)
    assert rel(x, f) < 1e-5
    assert rel(x, xo) < 1e-5


def test_errors(sp):
    import torch
    w = workload_ragged(N=8, I=1, S=20)
    with _plan(sp, w, 0) as p:
        with pytest.raises(sp.SpirecError) as e:
            sp.spirec_solve(p.h, None, 3, 8)
        assert e.value.code == sp.SPIREC_ESTATE
        bad = w["kx"].copy()
        bad[3] = 0.51
        with pytest.raises(sp.SpirecError) as e:
            sp.spirec_set_trajectory(p.h, bad, w["ky"])
        assert e.value.code == sp.SPIREC_EINVAL
        bad[3] = np.nan
        with pytest.raises(sp.SpirecError) as e:
            sp.spirec_set_trajectory(p.h, bad, w["ky"])
        assert e.value.code == sp.SPIREC_EINVAL
        with pytest.raises(sp.SpirecError) as e:
            sp.spirec_set_reg(p.h, -1.0, 0.1, 0.0, 0.1, 0)
        assert e.value.code == sp.SPIREC_EINVAL
    with pytest.raises(sp.SpirecError) as e:
        sp.Plan(8, 20, 10, 0, torch.cuda.current_stream().cuda_stream)  # M < 2N-1
    assert e.value.code == sp.SPIREC_EINVAL


def test_persistent_loop_matches_kernel_graph(sp, monkeypatch):
    """The persistent cooperative loop (default for power-of-two M) and the
    graph of stand-alone kernels run the same iteration; only their
    summation trees differ, so J agrees to 1e-5 and both match the oracle."""
    w = workload_c1()
    N, reg = w["N"], w["reg"]
    res = {}
    for mode in ("loop", "graph"):
        if mode == "graph":
            monkeypatch.setenv("SPIREC_NO_LOOP", "1")
        else:
            monkeypatch.delenv("SPIREC_NO_LOOP", raising=False)
        with _plan(sp, w, 0) as p:
            assert p.M == 64
            sp.spirec_set_data(p.h, w["s"])
            sp.spirec_set_reg(p.h, reg.lambda1, reg.alpha1, reg.lambda0, reg.alpha0, reg.kind)
            res[mode] = sp.spirec_solve(p.h, None, w["iters"], N)
    xo, Jo, _ = O.solve(w["kx"], w["ky"], w["s"], reg, np.zeros((N, N)), w["iters"])
    for mode in res:
        x, J = res[mode]
        assert rel(J, Jo) < 1e-5, mode
        assert rel(x, xo) < iter_tol(w, 0), (mode, rel(x, xo))
    assert rel(res["loop"][1], res["graph"][1]) < 1e-5


_LARGE = {}


def _large_case(N, I, S, seed):
    """A ragged large image and its 3-iteration oracle solve (cached)."""
    key = (N, I, S, seed)
    if key not in _LARGE:
        g = synth.rng(seed)
        f_true = synth.phantom(N, "ellipses_phase", g)
        kx, ky = synth.spiral(N, I, S, "variable")
        s = c64(synth.add_noise(O.forward(kx, ky, f_true), 30.0, g))
        reg = O.Reg(0.05, 0.05, 0.01, 0.1, O.PHI_HUBER)
        w = dict(N=N, kx=kx, ky=ky, f_true=f_true, s=s, reg=reg, iters=3)
        xo, Jo, _ = O.solve(kx, ky, s, reg, np.zeros((N, N)), 3)
        _LARGE[key] = (w, xo, Jo)
    return _LARGE[key]


# (N, M, interleaves, samples, seed): the M = 1024 loop (split 512-point
# column and row FFTs; N = 260 in 2-row blocks; N = 259 in 2-row blocks with
# a last block of one row and two blocks without a column group; N = 511 in
# 4-row blocks with a last block of three rows, so that some warp pairs of
# the row passes have no row), the M = 512 loop (radix-4 passes, 4-row
# groups), and M = 2048 and 4096, whose row caches do not fit a block: the
# solve falls back to the kernel graph, whose row and column passes split
# each row and column into 2 or 4 warp-sized 1024-point DFTs (N = 259 and 601
# leave a partial last row group of those passes)
LARGE_CASES = [(260, 1024, 3, 700, 21), (259, 1024, 3, 300, 53), (511, 1024, 2, 300, 57),
               (200, 512, 3, 500, 31), (520, 2048, 2, 400, 41),
               (600, 4096, 2, 300, 43), (259, 2048, 3, 300, 49), (601, 4096, 2, 300, 47)]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", LARGE_CASES, ids=lambda c: f"N{c[0]}_M{c[1]}")
def test_large_images_loop_and_graph(sp, monkeypatch, case, prec):
    """Persistent loop (or its fallback) and the stand-alone kernel graph
    against the oracle after 3 iterations, and against each other."""
    N, M, I, S, seed = case
    w, xo, Jo = _large_case(N, I, S, seed)
    reg = w["reg"]
    res = {}
    for mode in ("loop", "graph"):
        if mode == "graph":
            monkeypatch.setenv("SPIREC_NO_LOOP", "1")
        else:
            monkeypatch.delenv("SPIREC_NO_LOOP", raising=False)
        with _plan(sp, w, prec, M=M) as p:
            assert p.M == M
            sp.spirec_set_data(p.h, w["s"])
            sp.spirec_set_reg(p.h, reg.lambda1, reg.alpha1, reg.lambda0, reg.alpha0, reg.kind)
            res[mode] = sp.spirec_solve(p.h, None, w["iters"], N)
    for mode, (x, J) in res.items():
        assert np.all(np.diff(J) <= 1e-6 * J[0]), mode
        assert rel(J, Jo) < TOL[prec], mode
        assert rel(x, xo) < TOL[prec], mode
    assert rel(res["loop"][0], res["graph"][0]) < TOL[prec]


@pytest.mark.parametrize("prec", PRECISIONS)
def test_direct_mode_matches_oracle_and_toeplitz_mode(sp, prec):
    """SPIREC_MODE_DIRECT applies H^H H by the exact forward and adjoint
    NUDFT every iteration (the original formulation); it must reach the
    oracle's J history and iterates as the Toeplitz mode does."""
    w = workload_c1()
    N, reg, iters = w["N"], w["reg"], w["iters"]
    xo, Jo, _ = O.solve(w["kx"], w["ky"], w["s"], reg, np.zeros((N, N)), iters)
    res = {}
    for mode in (sp.SPIREC_MODE_TOEPLITZ, sp.SPIREC_MODE_DIRECT):
        with _plan(sp, w, prec) as p:
            sp.spirec_set_mode(p.h, mode)
            sp.spirec_set_data(p.h, w["s"])
            sp.spirec_set_reg(p.h, reg.lambda1, reg.alpha1, reg.lambda0, reg.alpha0, reg.kind)
            res[mode] = sp.spirec_solve(p.h, None, iters, N)
    x, J = res[sp.SPIREC_MODE_DIRECT]
    assert np.all(np.diff(J) <= 1e-6 * J[0])
    assert rel(J, Jo) < TOL[prec]
    assert rel(x, xo) < iter_tol(w, prec), rel(x, xo)
    assert rel(x, res[sp.SPIREC_MODE_TOEPLITZ][0]) < 2 * iter_tol(w, prec)


def test_direct_mode_from_x0_and_errors(sp):
    w = workload_ragged()
    N, reg = w["N"], w["reg"]
    g = synth.rng(8)
    x0 = (0.5 * w["f_true"] + 0.05 * synth.complex_normal(w["f_true"].shape, g)).astype(np.complex64)
    xo, Jo, _ = O.solve(w["kx"], w["ky"], w["s"], reg, c64(x0), 3)
    with _plan(sp, w, 0) as p:
        with pytest.raises(sp.SpirecError) as e:
            sp.spirec_set_mode(p.h, 7)
        assert e.value.code == sp.SPIREC_EINVAL
        sp.spirec_set_mode(p.h, sp.SPIREC_MODE_DIRECT)
        sp.spirec_set_data(p.h, w["s"])
        sp.spirec_set_reg(p.h, reg.lambda1, reg.alpha1, reg.lambda0, reg.alpha0, reg.kind)
        x, J = sp.spirec_solve(p.h, x0, 3, N)
        # switching back to the Toeplitz mode on the same plan
        sp.spirec_set_mode(p.h, sp.SPIREC_MODE_TOEPLITZ)
        xt, Jt = sp.spirec_solve(p.h, x0, 3, N)
    assert rel(J, Jo) < 1e-5 and rel(x, xo) < 1e-5
    assert rel(Jt, Jo) < 1e-5 and rel(xt, xo) < 1e-5
