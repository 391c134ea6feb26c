"""Failure detection, made to happen without faulting the GPU.

- An injected device-allocation failure: plan creation and the calls that
  allocate return SPIREC_ENOMEM, release what they had, and a plan made
  afterwards works.
- Bounded device waits that run out: a test stalls the persistent CG loop
  (one block waits for an arrival the grid never makes) or the tensor-core
  contractions (the MMA issuer waits on a barrier nothing completes), with a
  1 ms wait limit.  The kernels end early (the contractions after waiting for
  their own copies and MMAs and freeing their tensor memory), the plan
  reports SPIREC_ETIMEOUT, and after the limit is restored and the trajectory
  set again the same plan gives the oracle's results.
Nothing here traps, faults or leaves a kernel waiting without a bound."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0908_3252_gb300 import synth
from tests.helpers import c64, rel, workload_ragged

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0908_3252_gb300 import build, spirec
    build.build()
    spirec.load()
    yield spirec
    spirec.spirec_inject_alloc_failure(-1)
    spirec.spirec_inject_wait_stall(0)
    spirec.spirec_set_wait_limit_ns(0)


def test_injected_allocation_failure(sp):
    w = workload_ragged(N=24, I=2, S=150)
    L = w["kx"].shape[0]
    try:
        for n in (0, 1, 7, 15):
            sp.spirec_inject_alloc_failure(n)
            with pytest.raises(sp.SpirecError) as e:
                sp.Plan(w["N"], L, 0, 1, None, w["kx"], w["ky"])
            assert e.value.code == sp.SPIREC_ENOMEM
            assert "injected" in str(e.value)
        sp.spirec_inject_alloc_failure(-1)
        p = sp.Plan(w["N"], L, 0, 0, None, w["kx"], w["ky"])
        try:
            sp.spirec_inject_alloc_failure(0)
            with pytest.raises(sp.SpirecError) as e:
                sp.spirec_set_mode(p.h, sp.SPIREC_MODE_DIRECT)  # allocates its sample buffer
            assert e.value.code == sp.SPIREC_ENOMEM
            with pytest.raises(sp.SpirecError) as e:
                sp.spirec_set_minimiser(p.h, sp.SPIREC_MIN_HALF_QUADRATIC, 4)  # allocates its weights
            assert e.value.code == sp.SPIREC_ENOMEM
        finally:
            sp.spirec_inject_alloc_failure(-1)
            p.close()
    finally:
        sp.spirec_inject_alloc_failure(-1)
    reg = w["reg"]
    with sp.Plan(w["N"], L, 0, 0, None, w["kx"], w["ky"]) as p:
        sp.spirec_set_data(p.h, w["s"])
        sp.spirec_set_reg(p.h, reg.lambda1, reg.alpha1, reg.lambda0, reg.alpha0, reg.kind)
        x, J = sp.spirec_solve(p.h, None, 3, w["N"])
    xo, Jo, _ = O.solve(w["kx"], w["ky"], w["s"], reg, np.zeros((w["N"], w["N"])), 3)
    assert rel(x, xo) < 1e-5 and rel(J, Jo) < 1e-5


def _problem(N, I, S, seed):
    g = synth.rng(seed)
    kx, ky = synth.spiral(N, I, S)
    s = c64(synth.complex_normal(kx.shape[0], g))
    return kx, ky, s


@pytest.mark.parametrize("prec", [0, 1])
def test_loop_wait_runs_out(sp, prec):
    """N = 256, M = 512: a 64-block persistent loop, stalled."""
    N = 256
    kx, ky, s = _problem(N, 4, 1000, 31)
    with sp.Plan(N, kx.shape[0], 512, prec, None, kx, ky) as p:
        sp.spirec_set_data(p.h, s)
        sp.spirec_set_reg(p.h, 0.05, 0.05, 0.0, 0.05, 0)
        x_ref, J_ref = sp.spirec_solve(p.h, None, 5, N)
        try:
            sp.spirec_set_wait_limit_ns(1_000_000)
            sp.spirec_inject_wait_stall(sp.SPIREC_STALL_LOOP)
            with pytest.raises(sp.SpirecError) as e:
                sp.spirec_solve(p.h, None, 5, N)
            assert e.value.code == sp.SPIREC_ETIMEOUT
        finally:
            sp.spirec_inject_wait_stall(0)
            sp.spirec_set_wait_limit_ns(0)
        # the report stays until the trajectory is set again; then the plan
        # works as before, bitwise
        with pytest.raises(sp.SpirecError) as e:
            sp.spirec_sync(p.h)
        assert e.value.code == sp.SPIREC_ETIMEOUT
        sp.spirec_set_trajectory(p.h, kx, ky)
        sp.spirec_set_data(p.h, s)
        x, J = sp.spirec_solve(p.h, None, 5, N)
    assert np.array_equal(x, x_ref) and np.array_equal(J, J_ref)


@pytest.mark.parametrize("prec", [1, 2])
def test_contraction_waits_run_out(sp, prec):
    """The G build (k_tc_phase_gemm through spirec_set_trajectory) and the
    forward NUDFT (k_tc_forward through spirec_forward), each stalled."""
    N = 64
    kx, ky, s = _problem(N, 2, 2000, 32)
    x = c64(synth.complex_normal((N, N), synth.rng(33)))
    L = kx.shape[0]
    with sp.Plan(N, L, 0, prec, None, kx, ky) as p:
        sp.spirec_sync(p.h)
        try:
            sp.spirec_set_wait_limit_ns(1_000_000)
            sp.spirec_inject_wait_stall(sp.SPIREC_STALL_CONTRACTION)
            sp.spirec_set_trajectory(p.h, kx, ky)  # G is built in stream order
            with pytest.raises(sp.SpirecError) as e:
                sp.spirec_sync(p.h)
            assert e.value.code == sp.SPIREC_ETIMEOUT
        finally:
            sp.spirec_inject_wait_stall(0)
        sp.spirec_set_trajectory(p.h, kx, ky)  # a clean G, then the forward stalled
        sp.spirec_sync(p.h)
        try:
            sp.spirec_inject_wait_stall(sp.SPIREC_STALL_CONTRACTION)
            with pytest.raises(sp.SpirecError) as e:
                sp.spirec_forward(p.h, x)
            assert e.value.code == sp.SPIREC_ETIMEOUT
        finally:
            sp.spirec_inject_wait_stall(0)
            sp.spirec_set_wait_limit_ns(0)
        sp.spirec_set_trajectory(p.h, kx, ky)
        sp.spirec_sync(p.h)
        import torch
        G = torch.zeros((N, 2 * N - 1), dtype=torch.complex64, device="cuda:0")
        sp.spirec_gram_dev(p.h, G)
        torch.cuda.synchronize()
        G = G.cpu().numpy()
        y = sp.spirec_forward(p.h, x)
    assert rel(G, O.gram(kx, ky, N)[:, N - 1:].T) < 1e-3
    assert rel(y, O.forward(kx, ky, x)) < 1e-3


def test_stall_mask_is_checked(sp):
    with pytest.raises(sp.SpirecError) as e:
        sp.spirec_inject_wait_stall(8)
    assert e.value.code == sp.SPIREC_EINVAL


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("M", [0, 64])
def test_non_finite_criterion_is_reported(sp, prec, M):
    """Data with a NaN sample makes D, and so J, NaN; the host solve reads the
    last J back with its other copies and reports SPIREC_ENUMERIC (NaN only
    flows through arithmetic: no index or loop bound depends on data).  The
    same plan then solves finite data to the oracle's result.  M = 0 takes
    the plan's default size (the stand-alone kernels), M = 64 the persistent
    loop."""
    w = workload_ragged(N=24, I=2, S=150)
    reg = w["reg"]
    L = w["kx"].shape[0]
    bad = w["s"].copy()
    bad[L // 2] = np.complex64(complex(np.nan, 0.0))
    with sp.Plan(w["N"], L, M, prec, None, w["kx"], w["ky"]) as p:
        sp.spirec_set_reg(p.h, reg.lambda1, reg.alpha1, reg.lambda0, reg.alpha0, reg.kind)
        sp.spirec_set_data(p.h, bad)
        with pytest.raises(sp.SpirecError) as e:
            sp.spirec_solve(p.h, None, 3, w["N"])
        assert e.value.code == sp.SPIREC_ENUMERIC
        sp.spirec_set_data(p.h, w["s"])
        x, J = sp.spirec_solve(p.h, None, 3, w["N"])
    xo, Jo, _ = O.solve(w["kx"], w["ky"], w["s"], reg, np.zeros((w["N"], w["N"])), 3)
    tol = 1e-5 if prec == 0 else 1e-3
    assert rel(x, xo) < tol and rel(J, Jo) < tol
