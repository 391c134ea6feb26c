"""Pins of the FP32 rounding model (oracle/fp32_model.py), the control that
sets the tolerance of the FP32 path's iterates after many iterations.

With rounding and perturbations off it must be the FP64 minimiser of the
direct-form oracle (oracle.solve); with them on it must differ from it by
rounding-sized amounts early on (an FP16-sized or a missing rounding step
fails), store only FP32-representable vectors, and its perturbations must be
reproducible from their seed."""
import numpy as np
import pytest

from oracle import fp32_model as FM
from oracle import oracle as O
from oracle import toeplitz_cpu as TC
from tests.helpers import workload_c1, workload_ragged


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def _setup(w, M):
    N = w["N"]
    C = TC.kernel_spectrum(O.gram(w["kx"], w["ky"], N), N, M)
    D = O.adjoint(w["kx"], w["ky"], w["s"], N)
    ss = float(np.sum(np.abs(w["s"]) ** 2))
    return C, D, ss


@pytest.mark.parametrize("wname,M", [("c1", 64), ("ragged", 75)])
def test_fp64_limit_is_the_oracle(wname, M):
    """No rounding: the iterate and J history of oracle.solve (direct NUDFTs,
    Eq. CritLS) to FP64 rounding, so the model's steps (q1 from res,
    res += t T d, J from res) are the method's (section 3.3, Eq. NewCritLS)."""
    w = workload_c1() if wname == "c1" else workload_ragged()
    N, iters = w["N"], w["iters"]
    C, D, ss = _setup(w, M)
    x, J = FM.solve(C, D, ss, w["reg"], np.zeros((N, N)), iters, fp32=False)
    xo, Jo, _ = O.solve(w["kx"], w["ky"], w["s"], w["reg"], np.zeros((N, N)), iters)
    assert rel(x, xo) < 1e-9
    assert rel(J, Jo) < 1e-12


def test_rounding_is_single_precision():
    """After 3 iterations the rounded run stays within 1e-6 of FP64 (rounding
    to half precision would move it by ~1e-3), yet differs from it (a model
    that rounds nothing would not), and its iterate is FP32-representable."""
    w = workload_c1()
    N = w["N"]
    C, D, ss = _setup(w, 64)
    x64, _ = FM.solve(C, D, ss, w["reg"], np.zeros((N, N)), 3, fp32=False)
    x32, J32 = FM.solve(C, D, ss, w["reg"], np.zeros((N, N)), 3, fp32=True)
    assert 1e-10 < rel(x32, x64) < 1e-6
    assert np.array_equal(x32, FM.fl32(x32))
    assert np.all(np.diff(J32) <= 1e-9 * J32[0])


def test_perturbations_are_seeded():
    w = workload_ragged(N=16, I=2, S=100)
    C, D, ss = _setup(w, 32)
    a, _ = FM.solve(C, D, ss, w["reg"], np.zeros((16, 16)), 5, noise=1e-7, seed=3)
    b, _ = FM.solve(C, D, ss, w["reg"], np.zeros((16, 16)), 5, noise=1e-7, seed=3)
    c, _ = FM.solve(C, D, ss, w["reg"], np.zeros((16, 16)), 5, noise=1e-7, seed=4)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)
    sp = FM.spread(C, D, ss, w["reg"], np.zeros((16, 16)), 5, a, seeds=[3])
    assert len(sp) == 2 and sp[1] == 0.0
