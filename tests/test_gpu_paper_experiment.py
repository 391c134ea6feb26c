"""The paper's simulated experiment (section 4.1), with a stand-in for its
phantom (synth.vessels: two vessels, parabolic and blunt flow phase, on a
variable background, intensity scale ~255): 128 x 128, 6 spiral arms x 512
samples, 30 dB, Huber phi with the paper's hyperparameters lambda1 = 0.1,
alpha1 = 20, lambda0 = 0.5, alpha0 = 10, 50 iterations.

The GPU reconstruction is compared with the oracle's over all 50 iterations,
and the paper's two figures of merit (quadratic error in ROI1, variance in
ROI2) must favour the regularized reconstruction over the unregularized one,
as they do for the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0908_3252_gb300 import synth
from tests.helpers import c64, rel

pytestmark = pytest.mark.gpu

N, ITERS = 128, 50
PAPER = O.Reg(0.1, 20.0, 0.5, 10.0, O.PHI_HUBER)
UNREG = O.Reg(0.0, 20.0, 0.0, 10.0, O.PHI_HUBER)


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
def case():
    f, roi = synth.vessels(N)
    kx, ky = synth.spiral(N, 6, 512, "archimedean")
    s = c64(synth.add_noise(O.forward(kx, ky, f), 30.0, synth.rng(51)))
    xo, Jo, _ = O.solve(kx, ky, s, PAPER, np.zeros((N, N)), ITERS)
    return dict(f=f, roi=roi, kx=kx, ky=ky, s=s, xo=xo, Jo=Jo)


def _metrics(x, f, roi):
    err = float(np.sum(np.abs(x - f)[roi["roi1"]] ** 2) / np.sum(np.abs(f)[roi["roi1"]] ** 2))
    var = float(np.var(np.abs(x)[roi["roi2"]]))
    return err, var


def _solve(sp, c, reg, prec):
    import torch
    L = c["kx"].shape[0]
    with sp.Plan(N, L, 0, prec, torch.cuda.current_stream().cuda_stream, c["kx"], c["ky"]) as p:
        sp.spirec_set_data(p.h, c["s"])
        sp.spirec_set_reg(p.h, reg.lambda1, reg.alpha1, reg.lambda0, reg.alpha0, reg.kind)
        return sp.spirec_solve(p.h, None, ITERS, N)


@pytest.mark.parametrize("prec", [0, 1])
def test_paper_experiment_matches_oracle(sp, case, prec):
    x, J = _solve(sp, case, PAPER, prec)
    assert np.all(np.diff(J) <= 1e-6 * J[0])
    assert rel(J, case["Jo"]) < (1e-5 if prec == 0 else 1e-3)
    assert rel(x, case["xo"]) < 1e-3
    # the paper's figures of merit agree with the oracle's to three digits
    eg, vg = _metrics(x, case["f"], case["roi"])
    eo, vo = _metrics(case["xo"], case["f"], case["roi"])
    assert abs(eg - eo) <= 1e-3 * eo and abs(vg - vo) <= 1e-3 * vo


def test_regularization_improves_the_figures_of_merit(sp, case):
    x_reg, _ = _solve(sp, case, PAPER, 0)
    x_ls, _ = _solve(sp, case, UNREG, 0)
    e_reg, v_reg = _metrics(x_reg, case["f"], case["roi"])
    e_ls, v_ls = _metrics(x_ls, case["f"], case["roi"])
    assert e_reg < e_ls
    assert v_reg < v_ls
