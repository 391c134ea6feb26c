"""Many reconstructions on one GPU: the request loop (continuous batching)
and the batched solve, through the C ABI.

The central property: each request's result is the same when it runs alone
and when it runs in a mix with others on the same GPU (launch shapes and
summation orders depend only on the request's own sizes, so the results are
identical, not merely close)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0908_3252_gb300 import synth
from tests.helpers import c64, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0908_3252_gb300 import build, spirec
    build.build()
    spirec.load()
    return spirec


def _requests(n, seed=11):
    g = synth.rng(seed)
    reqs = []
    for i in range(n):
        N = [24, 32, 40, 48, 64][i % 5]
        I, S = 2 + i % 3, 200 + 37 * i
        kx, ky = synth.spiral(N, I, S, "variable" if i % 2 else "archimedean")
        f = synth.phantom(N, "ellipses_phase", g)
        s = c64(synth.add_noise(O.forward(kx, ky, f), 30.0, g))
        reqs.append(dict(N=N, kx=kx, ky=ky, s=s, lambda1=0.02 + 0.01 * i, alpha1=0.05, lambda0=0.0,
                         alpha0=0.05, phi=0, iters=20))
    return reqs


def _submit(sp, srv, r):
    return sp.spirec_server_submit(srv, r["N"], r["kx"], r["ky"], r["s"], r["lambda1"], r["alpha1"],
                                   r["lambda0"], r["alpha0"], r["phi"], r["iters"])


@pytest.mark.parametrize("prec", [0, 1])
def test_results_alone_equal_results_in_mix(sp, prec):
    reqs = _requests(10)
    alone = []
    srv = sp.spirec_server_create(8 << 30, 1, prec)
    try:
        for r in reqs:
            t = _submit(sp, srv, r)
            alone.append(sp.spirec_server_wait(srv, t, r["N"]))
    finally:
        sp.spirec_server_destroy(srv)
    srv = sp.spirec_server_create(8 << 30, 4, prec)
    try:
        tickets = [_submit(sp, srv, r) for r in reqs]           # all queued at once
        mixed = [sp.spirec_server_wait(srv, t, r["N"]) for t, r in zip(tickets, reqs)]
        st = sp.spirec_server_stats(srv)
    finally:
        sp.spirec_server_destroy(srv)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert 0 < st["p50_s"] <= st["p99_s"]
    for (xa, Ja, _), (xm, Jm, _) in zip(alone, mixed):
        assert np.array_equal(xa, xm)
        assert Ja == Jm
    # and the first request against the oracle
    r = reqs[0]
    xo, Jo, _ = O.solve(r["kx"], r["ky"], r["s"], O.Reg(r["lambda1"], r["alpha1"], r["lambda0"], r["alpha0"],
                                                       r["phi"]), np.zeros((r["N"], r["N"])), r["iters"])
    assert abs(alone[0][1] - Jo[-1]) < (1e-5 if prec == 0 else 1e-3) * Jo[0]
    assert rel(alone[0][0], xo) < 1e-3


def test_admission_by_footprint(sp):
    """A budget that holds one plan: two slots still complete every request,
    one at a time; a request larger than the budget is refused."""
    reqs = _requests(4, seed=12)
    srv = sp.spirec_server_create(4 << 20, 2, 0)
    try:
        tickets = [_submit(sp, srv, r) for r in reqs]
        for t, r in zip(tickets, reqs):
            x, J, lat = sp.spirec_server_wait(srv, t, r["N"])
            assert np.isfinite(J) and lat > 0
        big = dict(reqs[0])
        N = 512
        big["N"] = N
        big["kx"], big["ky"] = synth.spiral(N, 4, 2048)
        big["s"] = np.zeros(big["kx"].shape[0], np.complex64)
        with pytest.raises(sp.SpirecError) as e:
            _submit(sp, srv, big)
        assert e.value.code == sp.SPIREC_EBUSY
    finally:
        sp.spirec_server_destroy(srv)


def test_wait_timeout_and_request_errors(sp):
    reqs = _requests(2, seed=13)
    srv = sp.spirec_server_create(8 << 30, 1, 0)
    try:
        r = dict(reqs[0])
        r["iters"] = 400
        t = _submit(sp, srv, r)
        with pytest.raises(sp.SpirecError) as e:
            sp.spirec_server_wait(srv, t, r["N"], timeout_ms=0)
        assert e.value.code == sp.SPIREC_ETIMEOUT
        sp.spirec_server_wait(srv, t, r["N"])  # the request was not lost
        bad = dict(reqs[1])
        bad["kx"] = bad["kx"].copy()
        bad["kx"][5] = 0.75
        t = _submit(sp, srv, bad)
        with pytest.raises(sp.SpirecError) as e:
            sp.spirec_server_wait(srv, t, bad["N"])
        assert e.value.code == sp.SPIREC_EINVAL
        # the loop keeps serving after a failed request
        t = _submit(sp, srv, reqs[1])
        sp.spirec_server_wait(srv, t, reqs[1]["N"])
    finally:
        sp.spirec_server_destroy(srv)


def test_batch_solve_equals_single_solves(sp):
    import torch
    reqs = _requests(4, seed=14)
    plans, outs, Js, keep = [], [], [], []
    try:
        for r in reqs:
            st = torch.cuda.Stream()
            p = sp.Plan(r["N"], r["kx"].shape[0], 0, 1, st.cuda_stream)
            kx = torch.from_numpy(r["kx"]).cuda()
            ky = torch.from_numpy(r["ky"]).cuda()
            s = torch.from_numpy(r["s"].astype(np.complex64)).cuda()
            keep += [kx, ky, s]  # alive until the asynchronous work has run
            torch.cuda.synchronize()
            sp.spirec_set_trajectory_dev(p.h, kx, ky)
            sp.spirec_set_data_dev(p.h, s)
            sp.spirec_set_reg(p.h, r["lambda1"], r["alpha1"], r["lambda0"], r["alpha0"], r["phi"])
            plans.append((p, st))
            outs.append(torch.zeros((r["N"], r["N"]), dtype=torch.complex64, device="cuda"))
            Js.append(torch.zeros(21, dtype=torch.float64, device="cuda"))
        torch.cuda.synchronize()
        sp.spirec_batch_solve([p.h for p, _ in plans], outs, 20, J_hist=Js)
        torch.cuda.synchronize()
        for (p, _), r, o in zip(plans, reqs, outs):
            x, J = sp.spirec_solve(p.h, None, 20, r["N"])
            assert np.array_equal(x, o.cpu().numpy())
    finally:
        for p, _ in plans:
            p.close()


def test_idle_plans_are_released_for_a_larger_request(sp):
    """Two idle workers each keep the plan of their last request; the next
    request fits the budget alone but not beside either plan.  The workers
    must release their idle plans for it (before, no worker admitted it and
    the queue stalled, as nothing was running to wake them)."""
    g = synth.rng(21)

    def req(N, I, S):
        kx, ky = synth.spiral(N, I, S)
        return dict(N=N, kx=kx, ky=ky, s=c64(synth.complex_normal(kx.shape[0], g)), lambda1=0.05, alpha1=0.05,
                    lambda0=0.0, alpha0=0.05, phi=0, iters=5)

    a, b, c = req(48, 2, 500), req(64, 2, 600), req(160, 8, 2048)
    ba = sp.spirec_server_plan_bytes(a["N"], a["kx"].shape[0], 0)[0]
    bb = sp.spirec_server_plan_bytes(b["N"], b["kx"].shape[0], 0)[0]
    bc = sp.spirec_server_plan_bytes(c["N"], c["kx"].shape[0], 0)[0]
    assert bc > ba + bb
    budget = bc + (1 << 16)  # c fits alone, not beside a or b
    srv = sp.spirec_server_create(budget, 2, 0)
    try:
        ta = _submit(sp, srv, a)
        tb = _submit(sp, srv, b)
        sp.spirec_server_wait(srv, ta, a["N"], timeout_ms=60000)
        sp.spirec_server_wait(srv, tb, b["N"], timeout_ms=60000)
        tc = _submit(sp, srv, c)
        x, J, _ = sp.spirec_server_wait(srv, tc, c["N"], timeout_ms=60000)
        assert np.isfinite(J)
        st = sp.spirec_server_stats(srv)
        assert st["completed"] == 3 and st["failed"] == 0
    finally:
        sp.spirec_server_destroy(srv)


@pytest.mark.parametrize("prec", [0, 1])
def test_footprint_estimate_covers_the_plan(sp, prec):
    """The request loop admits by spirec_server_plan_bytes: it must cover
    every buffer a plan of that shape allocates through a served request's
    calls (trajectory, data, penalty, solve)."""
    g = synth.rng(22)
    for N, L in [(2, 1), (24, 333), (64, 5000), (100, 20000), (192, 8192), (256, 70000), (384, 200000)]:
        nbytes, M = sp.spirec_server_plan_bytes(N, L, prec)
        kx, ky = synth.uniform_k(L, g)
        with sp.Plan(N, L, M, prec, None, kx, ky) as p:
            sp.spirec_set_data(p.h, c64(synth.complex_normal(L, g)))
            sp.spirec_set_reg(p.h, 0.05, 0.05, 0.0, 0.05, 0)
            sp.spirec_solve(p.h, None, 1, N)
            used = sp.spirec_plan_info(p.h)["device_bytes"]
        assert used <= nbytes, (N, L, used, nbytes)


def test_concurrent_persistent_loops_all_complete(sp):
    """Eight slots of the largest loop grids (N = 384 to 512: 96 to 128
    one-SM blocks each, so no two fit the device together): every solve
    must complete (no loop left waiting for blocks another loop holds) and
    equal its result alone."""
    g = synth.rng(23)
    reqs = []
    for i in range(8):
        N = [384, 448, 512, 512][i % 4]
        kx, ky = synth.spiral(N, 2, 700 + 50 * i)
        reqs.append(dict(N=N, kx=kx, ky=ky, s=c64(synth.complex_normal(kx.shape[0], g)), lambda1=0.05,
                         alpha1=0.05, lambda0=0.0, alpha0=0.05, phi=0, iters=10))
    srv = sp.spirec_server_create(64 << 30, 8, 1)
    try:
        tickets = [_submit(sp, srv, r) for r in reqs]
        mixed = [sp.spirec_server_wait(srv, t, r["N"], timeout_ms=120000) for t, r in zip(tickets, reqs)]
        st = sp.spirec_server_stats(srv)
    finally:
        sp.spirec_server_destroy(srv)
    assert st["completed"] == 8 and st["failed"] == 0
    srv = sp.spirec_server_create(64 << 30, 1, 1)
    try:
        for r, (xm, Jm, _) in zip(reqs[:4], mixed[:4]):
            xa, Ja, _ = sp.spirec_server_wait(srv, _submit(sp, srv, r), r["N"], timeout_ms=120000)
            assert np.array_equal(xa, xm) and Ja == Jm
    finally:
        sp.spirec_server_destroy(srv)
