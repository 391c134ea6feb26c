"""The host-pointer operator calls of the C ABI (spirec_forward,
spirec_adjoint, spirec_gram_apply, spirec_objective_grad) against the FP64
oracle, at the tolerances of the device-pointer parity tests: H x (Eq.
ModDirect), H^H y (Eq. AnnMatGD), T x = H^H H x (Appendix B) and J, grad J
(Eq. NewCritLS plus the penalty of section 3.3)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0908_3252_gb300 import synth
from tests.helpers import c64, rel, workload_c1, workload_ragged

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-3, 2: 1e-3}


@pytest.fixture(scope="module")
def sp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0908_3252_gb300 import build, spirec
    build.build()
    spirec.load()
    return spirec


def _w(name):
    return workload_c1() if name == "c1" else workload_ragged()


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("wname", ["c1", "ragged"])
def test_forward_and_adjoint(sp, prec, wname):
    w = _w(wname)
    N, L = w["N"], w["kx"].shape[0]
    g = synth.rng(61)
    x = c64(synth.complex_normal((N, N), g))
    y = c64(synth.complex_normal(L, g))
    with sp.Plan(N, L, 0, prec, None, w["kx"], w["ky"]) as p:
        Hx = sp.spirec_forward(p.h, x)
        Hy = sp.spirec_adjoint(p.h, y)
        # twice in a row: the staging buffers leave nothing behind
        Hx2 = sp.spirec_forward(p.h, x)
        Hy2 = sp.spirec_adjoint(p.h, y)
    assert rel(Hx, O.forward(w["kx"], w["ky"], x)) < TOL[prec]
    assert rel(Hy, O.adjoint(w["kx"], w["ky"], y, N)) < TOL[prec]
    assert np.array_equal(Hx, Hx2) and np.array_equal(Hy, Hy2)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("wname", ["c1", "ragged"])
def test_gram_apply(sp, prec, wname):
    w = _w(wname)
    N = w["N"]
    x = c64(synth.complex_normal((N, N), synth.rng(62)))
    with sp.Plan(N, w["kx"].shape[0], 0, prec, None, w["kx"], w["ky"]) as p:
        Tx = sp.spirec_gram_apply(p.h, x)
    want = O.adjoint(w["kx"], w["ky"], O.forward(w["kx"], w["ky"], x), N)
    assert rel(Tx, want) < TOL[prec]


@pytest.mark.parametrize("kind", [O.PHI_HUBER, O.PHI_HYPERBOLIC, O.PHI_QUADRATIC])
def test_objective_grad(sp, kind):
    """J and grad J are differences of far larger terms in the rewritten form;
    the bound is stated against those terms (as in test_gpu_parity)."""
    w = workload_ragged(kind=kind)
    N, reg = w["N"], w["reg"]
    x = c64(w["f_true"] + 0.1 * synth.complex_normal((N, N), synth.rng(63)))
    with sp.Plan(N, w["kx"].shape[0], 0, 0, None, w["kx"], w["ky"]) as p:
        with pytest.raises(sp.SpirecError) as e:
            sp.spirec_objective_grad(p.h, x)
        assert e.value.code == sp.SPIREC_ESTATE
        sp.spirec_set_data(p.h, w["s"])
        sp.spirec_set_reg(p.h, reg.lambda1, reg.alpha1, reg.lambda0, reg.alpha0, reg.kind)
        J, gr = sp.spirec_objective_grad(p.h, x)
    kx, ky, s = w["kx"], w["ky"], w["s"]
    D = O.adjoint(kx, ky, s, N)
    Tx = O.adjoint(kx, ky, O.forward(kx, ky, x), N)
    gR = O.penalty_grad(x, reg)
    J_terms = np.sum(np.abs(s) ** 2) + 2 * abs(np.vdot(x, D)) + abs(np.vdot(x, Tx)) + O.penalty(x, reg)
    g_terms = 2 * np.linalg.norm(Tx) + 2 * np.linalg.norm(D) + np.linalg.norm(gR)
    assert np.linalg.norm(gr - O.gradient(kx, ky, s, x, reg)) < 1e-5 * g_terms
    assert abs(J - O.objective(kx, ky, s, x, reg)) < 1e-5 * J_terms


def test_operator_calls_need_a_trajectory(sp):
    p = sp.Plan(8, 20, 0, 0)
    try:
        with pytest.raises(sp.SpirecError) as e:
            sp.spirec_forward(p.h, np.zeros((8, 8), np.complex64))
        assert e.value.code == sp.SPIREC_ESTATE
        with pytest.raises(sp.SpirecError) as e:
            sp.spirec_gram_apply(p.h, np.zeros((8, 8), np.complex64))
        assert e.value.code == sp.SPIREC_ESTATE
    finally:
        p.close()
