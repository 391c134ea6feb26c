"""End-to-end error of every precision against the FP64 oracle on the
benchmark's own workload: N = 512, Archimedean spiral 32 x 4096
(L = 131072), M = 1024, edges-and-texture phantom, 30 dB, Huber phi
(alpha 0.05, lambda1 0.05), 50 iterations from zero.

The FP64 reference is the paper's rewritten criterion solved in FP64
(oracle/toeplitz_cpu.py, itself pinned to the direct-form oracle to 3e-11),
with G and D from the matrix-product form of the oracle's sums
(oracle/factored.py, pinned to the direct sums); the data are simulated by the
same FP64 forward model.  Beside each GPU path's distance stands the FP32
rounding model's (oracle/fp32_model.py): the spread an FP32 implementation of
the method shows on this problem.  Each path must land within its target
(1e-5 FP32, 1e-3 mixed) or within 3 x that spread, whichever is larger; the
J history within 1e-5 of ||s||^2 (the scale of the terms the rewritten
criterion cancels) or 3 x the model's largest J difference, whichever is
larger (PR+ restarts that rounding flips make the histories part for a few
iterations and meet again, in the model as on the GPU)."""
import numpy as np
import pytest

from oracle import factored as F
from oracle import fp32_model as FM
from oracle import oracle as O
from oracle import toeplitz_cpu as TC
from paper_0908_3252_gb300 import synth
from tests.helpers import OPERATOR_NOISE, c64, rel

pytestmark = pytest.mark.gpu

N, I, S, M, ITERS = 512, 32, 4096, 1024, 50
TARGET = {0: 1e-5, 1: 1e-3, 2: 1e-3}


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
def problem():
    g = synth.rng(3)
    f_true = synth.phantom(N, "edges_texture", g)
    kx, ky = synth.spiral(N, I, S, "archimedean")
    s = c64(synth.add_noise(F.forward(kx, ky, f_true), 30.0, g))
    reg = O.Reg(0.05, 0.05, 0.0, 0.05, O.PHI_HUBER)
    C, D, ss = TC.problem_fp64(kx, ky, s, N, M)
    x0 = np.zeros((N, N))
    x64, J64 = TC.solve(C, D, ss, reg, x0, ITERS)
    spread, jspread = FM.deviations(C, D, ss, reg, x0, ITERS, x64, J64, noise=OPERATOR_NOISE, seeds=[0, 1])
    return dict(kx=kx, ky=ky, s=s, reg=reg, ss=ss, x64=x64, J64=J64, spread=spread, jspread=jspread,
                f_true=f_true)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_end_to_end_error_vs_fp64(sp, problem, prec):
    pb = problem
    reg = pb["reg"]
    with sp.Plan(N, pb["kx"].shape[0], M, prec, None, pb["kx"], pb["ky"]) as p:
        sp.spirec_set_data(p.h, pb["s"])
        sp.spirec_set_reg(p.h, reg.lambda1, reg.alpha1, reg.lambda0, reg.alpha0, reg.kind)
        x, J = sp.spirec_solve(p.h, None, ITERS, N)
    err = rel(x, pb["x64"])
    jerr = float(np.max(np.abs(J - pb["J64"])))
    tol = max(TARGET[prec], 3.0 * max(pb["spread"]))
    jtol = max(1e-5 * pb["ss"], 3.0 * max(pb["jspread"]))
    print(f"precision {prec}: iterate {err:.3e} from FP64 (FP32 model "
          f"{', '.join('%.2e' % v for v in pb['spread'])}; tolerance {tol:.2e}); "
          f"J history {jerr / pb['ss']:.2e} of ||s||^2 (FP32 model "
          f"{', '.join('%.2e' % (v / pb['ss']) for v in pb['jspread'])}; tolerance {jtol / pb['ss']:.2e}); "
          f"final J {abs(J[-1] - pb['J64'][-1]) / pb['J64'][-1]:.2e} relative")
    assert np.all(np.diff(J) <= 1e-6 * J[0])
    assert err < tol
    assert jerr < jtol
