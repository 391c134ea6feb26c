"""The half-quadratic minimiser on the GPU (spirec_set_minimiser) against the
FP64 half-quadratic oracle (oracle/halfquad.py), through the C ABI.

Tolerances as in test_gpu_parity: the J history to 1e-5 (FP32 contraction)
or 1e-3 (FP16x3 / BF16x3) relative L2; iterates after a few outer steps to
1e-4 / 1e-3 (FP32 linear CG compounds the rounding of its T applies)."""
import numpy as np
import pytest

from oracle import halfquad as HQ
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


def _gpu_hq(sp, w, prec, outer, inner, x0=None, mode=0, M=0):
    with _plan(sp, w, prec, M) as p:
        sp.spirec_set_mode(p.h, mode)
        sp.spirec_set_minimiser(p.h, sp.SPIREC_MIN_HALF_QUADRATIC, inner)
        return sp.spirec_solve(p.h, x0, outer, w["N"])


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("wname", ["c1", "ragged"])
def test_matches_the_oracle(sp, prec, wname):
    w = workload_c1() if wname == "c1" else workload_ragged()
    N = w["N"]
    x, J = _gpu_hq(sp, w, prec, 6, 4)
    xo, Jo = HQ.solve(w["kx"], w["ky"], w["s"], w["reg"], np.zeros((N, N)), 6, 4)
    assert J.shape == (7,)
    assert rel(J, Jo) < TOL[prec]
    assert rel(x, xo) < XTOL[prec]


def test_from_x0_and_quadratic_phi(sp):
    """A start point, and quadratic phi (constant weights: one outer step is
    plain linear CG on the normal equations), run to convergence.  Part-way
    through, linear CG on this underdetermined problem (L < N^2) is
    sensitive to rounding: with weights 0.05 / 0.02 and 25 steps, the oracle
    itself moves by 2.7e-3 in x when each of its T applies is perturbed by
    1e-7 relative noise, while J moves by 5e-5.  With 0.5 / 0.2 and 25 steps,
    CG has converged and the same perturbation moves x by 4e-6."""
    w = workload_ragged()
    N = w["N"]
    g = synth.rng(4)
    x0 = (0.5 * w["f_true"] + 0.05 * synth.complex_normal((N, N), g)).astype(np.complex64)
    x, J = _gpu_hq(sp, w, 0, 4, 5, x0=x0)
    xo, Jo = HQ.solve(w["kx"], w["ky"], w["s"], w["reg"], c64(x0), 4, 5)
    assert rel(J, Jo) < 1e-5 and rel(x, xo) < 1e-4
    wq = dict(w, reg=O.Reg(0.5, 1.0, 0.2, 1.0, O.PHI_QUADRATIC))
    x, J = _gpu_hq(sp, wq, 0, 1, 25)
    xo, Jo = HQ.solve(wq["kx"], wq["ky"], wq["s"], wq["reg"], np.zeros((N, N)), 1, 25)
    assert rel(J, Jo) < 1e-5 and rel(x, xo) < 1e-4


@pytest.mark.parametrize("prec", [0, 1])
def test_criterion_never_increases(sp, prec):
    w = workload_c1()
    _, J = _gpu_hq(sp, w, prec, 25, 5)
    assert np.all(np.isfinite(J))
    assert np.all(np.diff(J) <= 1e-6 * J[0])
    assert J[-1] < 0.1 * J[0]


def test_direct_mode_equals_toeplitz_mode(sp):
    """The inner T applies by the exact NUDFT pair instead of the FFT
    convolution: the same iterates up to rounding, and the oracle's."""
    w = workload_ragged()
    N = w["N"]
    xt, Jt = _gpu_hq(sp, w, 0, 5, 4, mode=0)
    xd, Jd = _gpu_hq(sp, w, 0, 5, 4, mode=1)
    xo, Jo = HQ.solve(w["kx"], w["ky"], w["s"], w["reg"], np.zeros((N, N)), 5, 4)
    assert rel(xd, xt) < 1e-4 and rel(Jd, Jt) < 1e-5
    assert rel(Jd, Jo) < 1e-5


def test_larger_image(sp):
    """200 x 200 with M = 512 (several tiles of every kernel)."""
    N = 200
    g = synth.rng(9)
    f = synth.phantom(N, "ellipses_phase", g)
    kx, ky = synth.spiral(N, 3, 500, "variable")
    s = c64(synth.add_noise(O.forward(kx, ky, f), 30.0, g))
    w = dict(N=N, kx=kx, ky=ky, s=s, reg=O.Reg(0.05, 0.05, 0.01, 0.1, O.PHI_HUBER))
    x, J = _gpu_hq(sp, w, 1, 3, 3, M=512)
    xo, Jo = HQ.solve(kx, ky, s, w["reg"], np.zeros((N, N)), 3, 3)
    assert rel(J, Jo) < 1e-3 and rel(x, xo) < 1e-3


def test_zero_outer_steps_and_switching_back(sp):
    """iters = 0 gives J(x0) alone; switching back to PR+ CG on the same plan
    gives what a new plan gives."""
    w = workload_c1()
    N = w["N"]
    with _plan(sp, w, 0) as p:
        sp.spirec_set_minimiser(p.h, sp.SPIREC_MIN_HALF_QUADRATIC, 3)
        x0, J0 = sp.spirec_solve(p.h, None, 0, N)
        sp.spirec_solve(p.h, None, 5, N)
        sp.spirec_set_minimiser(p.h, sp.SPIREC_MIN_PRCG)
        x1, J1 = sp.spirec_solve(p.h, None, 10, N)
    with _plan(sp, w, 0) as q:
        x2, J2 = sp.spirec_solve(q.h, None, 10, N)
    assert np.array_equal(x1, x2) and np.array_equal(J1, J2)
    assert np.all(x0 == 0) and J0.shape == (1,)
    assert abs(J0[0] - O.objective(w["kx"], w["ky"], w["s"], np.zeros((N, N)), w["reg"])) < 1e-5 * J0[0]


def test_bad_arguments(sp):
    w = workload_c1()
    with _plan(sp, w, 0) as p:
        for kind, inner in [(3, 3), (-1, 3), (1, 0), (1, 1001)]:
            with pytest.raises(sp.SpirecError) as e:
                sp.spirec_set_minimiser(p.h, kind, inner)
            assert e.value.code == sp.SPIREC_EINVAL
