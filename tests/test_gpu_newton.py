"""The truncated Newton minimiser on the GPU (spirec_set_minimiser with
SPIREC_MIN_NEWTON) against the FP64 Newton oracle (oracle/newton.py), through
the C ABI.

Tolerances as in test_gpu_parity: the J history to 1e-5 (FP32 contraction)
or 1e-3 (FP16x3 / BF16x3) relative L2, the iterates to 1e-4 / 1e-3.  On the
workloads used, the oracle's iterates move by about 6e-8 under a 1e-7
relative perturbation of the data and by 3e-6 (Huber, the ragged workload)
when each of its Hessian applies is perturbed by 1e-7 relative noise, so FP32
rounding stays inside 1e-4."""
import numpy as np
import pytest

from oracle import newton as NT
from oracle import oracle as O
from paper_0908_3252_gb300 import synth
from tests.helpers import c64, rel, workload_c1, workload_ragged

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-3, 2: 1e-3}
XTOL = {0: 1e-4, 1: 1e-3, 2: 1e-3}


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
    p = sp.Plan(w["N"], w["kx"].shape[0], M, prec, torch.cuda.current_stream().cuda_stream, w["kx"], w["ky"])
    sp.spirec_set_data(p.h, w["s"])
    r = w["reg"]
    sp.spirec_set_reg(p.h, r.lambda1, r.alpha1, r.lambda0, r.alpha0, r.kind)
    return p


def _gpu_nt(sp, w, prec, outer, inner, x0=None, mode=0, M=0):
    with _plan(sp, w, prec, M) as p:
        sp.spirec_set_mode(p.h, mode)
        sp.spirec_set_minimiser(p.h, sp.SPIREC_MIN_NEWTON, inner)
        return sp.spirec_solve(p.h, x0, outer, w["N"])


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("wname", ["c1", "ragged"])
def test_matches_the_oracle(sp, prec, wname):
    w = workload_c1() if wname == "c1" else workload_ragged()
    N = w["N"]
    x, J = _gpu_nt(sp, w, prec, 6, 4)
    xo, Jo = NT.solve(w["kx"], w["ky"], w["s"], w["reg"], np.zeros((N, N)), 6, 4)
    assert J.shape == (7,)
    assert rel(J, Jo) < TOL[prec]
    assert rel(x, xo) < XTOL[prec]


@pytest.mark.parametrize("kind,reg,outer,inner", [
    (O.PHI_HYPERBOLIC, O.Reg(0.2, 0.1, 0.05, 0.2, O.PHI_HYPERBOLIC), 4, 5),
    (O.PHI_QUADRATIC, O.Reg(0.5, 1.0, 0.2, 1.0, O.PHI_QUADRATIC), 2, 25)])
def test_from_x0_and_other_penalties(sp, kind, reg, outer, inner):
    """A start point; the hyperbolic phi on both terms and the quadratic phi
    (the rank-one Hessian part vanishes there, and the first step with 25
    inner steps has converged).  The weights keep the Newton systems well
    conditioned: with lambda1 = 0.05, lambda0 = 0.02 (the ragged workload's)
    and quadratic phi, the oracle's iterate moves by 3e-3 when each of its
    Hessian applies is perturbed by 1e-7 relative noise (linear CG on a
    nearly singular system, L < N^2); with these weights it moves by 1.4e-5
    (hyperbolic) and 2e-10 (quadratic) under 1e-6 noise."""
    w = dict(workload_ragged(kind=kind), reg=reg)
    N = w["N"]
    g = synth.rng(6)
    x0 = (0.5 * w["f_true"] + 0.05 * synth.complex_normal((N, N), g)).astype(np.complex64)
    x, J = _gpu_nt(sp, w, 0, outer, inner, x0=x0)
    xo, Jo = NT.solve(w["kx"], w["ky"], w["s"], w["reg"], c64(x0), outer, inner)
    assert rel(J, Jo) < 1e-5 and rel(x, xo) < 1e-4


@pytest.mark.parametrize("prec", [0, 1])
def test_criterion_never_increases(sp, prec):
    w = workload_c1()
    _, J = _gpu_nt(sp, w, prec, 20, 6)
    assert np.all(np.isfinite(J))
    assert np.all(np.diff(J) <= 1e-6 * J[0])
    assert J[-1] < 0.1 * J[0]


def test_direct_mode_equals_toeplitz_mode(sp):
    """The inner T applies by the exact NUDFT pair instead of the FFT
    convolution: the same iterates up to rounding, and the oracle's."""
    w = workload_ragged()
    N = w["N"]
    xt, Jt = _gpu_nt(sp, w, 0, 4, 4, mode=0)
    xd, Jd = _gpu_nt(sp, w, 0, 4, 4, mode=1)
    xo, Jo = NT.solve(w["kx"], w["ky"], w["s"], w["reg"], np.zeros((N, N)), 4, 4)
    assert rel(xd, xt) < 1e-4 and rel(Jd, Jt) < 1e-5
    assert rel(Jd, Jo) < 1e-5


def test_larger_image_graph_path(sp):
    """200 x 200 with M = 512, and 300 x 300 with M = 2048 (the split row and
    column passes apply T)."""
    for N, M in [(200, 512), (300, 2048)]:
        g = synth.rng(N)
        f = synth.phantom(N, "ellipses_phase", g)
        kx, ky = synth.spiral(N, 3, 400, "variable")
        s = c64(synth.add_noise(O.forward(kx, ky, f), 30.0, g))
        w = dict(N=N, kx=kx, ky=ky, s=s, reg=O.Reg(0.05, 0.05, 0.01, 0.1, O.PHI_HUBER))
        x, J = _gpu_nt(sp, w, 1, 2, 3, M=M)
        xo, Jo = NT.solve(kx, ky, s, w["reg"], np.zeros((N, N)), 2, 3)
        assert rel(J, Jo) < 1e-3 and rel(x, xo) < 1e-3


def test_switching_minimisers_and_repeatability(sp):
    """Newton after the half-quadratic minimiser on one plan gives what a new
    plan gives, bitwise; iters = 0 gives J(x0) alone."""
    w = workload_c1()
    N = w["N"]
    with _plan(sp, w, 0) as p:
        sp.spirec_set_minimiser(p.h, sp.SPIREC_MIN_HALF_QUADRATIC, 3)
        sp.spirec_solve(p.h, None, 3, N)
        sp.spirec_set_minimiser(p.h, sp.SPIREC_MIN_NEWTON, 4)
        x0, J0 = sp.spirec_solve(p.h, None, 0, N)
        x1, J1 = sp.spirec_solve(p.h, None, 5, N)
    with _plan(sp, w, 0) as q:
        sp.spirec_set_minimiser(q.h, sp.SPIREC_MIN_NEWTON, 4)
        x2, J2 = sp.spirec_solve(q.h, None, 5, N)
    assert np.array_equal(x1, x2) and np.array_equal(J1, J2)
    assert np.all(x0 == 0) and J0.shape == (1,)


def test_bad_arguments(sp):
    w = workload_c1()
    with _plan(sp, w, 0) as p:
        for kind, inner in [(3, 3), (sp.SPIREC_MIN_NEWTON, 0), (sp.SPIREC_MIN_NEWTON, 1001)]:
            with pytest.raises(sp.SpirecError) as e:
                sp.spirec_set_minimiser(p.h, kind, inner)
            assert e.value.code == sp.SPIREC_EINVAL
