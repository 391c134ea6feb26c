"""The autotuner on the GPU: every value it may choose gives results within
the tolerances against the FP64 oracle, a tuned plan holds the same state as
a new plan of its shape, and captured iteration graphs follow the table."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0908_3252_gb300 import synth
from tests.helpers import c64, empty_c64, from_dev, rel

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
    spirec.spirec_tune_clear()
    yield spirec
    spirec.spirec_tune_clear()


@pytest.fixture(autouse=True)
def _empty_table(sp):
    sp.spirec_tune_clear()
    yield
    sp.spirec_tune_clear()


def _workload(N=48, I=3, S=600, seed=21):
    g = synth.rng(seed)
    f = synth.phantom(N, "ellipses_phase", g)
    kx, ky = synth.spiral(N, I, S, "variable")
    s = c64(synth.add_noise(O.forward(kx, ky, f), 30.0, g))
    reg = O.Reg(0.05, 0.05, 0.01, 0.1, O.PHI_HUBER)
    return dict(N=N, kx=kx, ky=ky, s=s, reg=reg)


def _plan(sp, w, prec, M=0):
    import torch
    p = sp.Plan(w["N"], w["kx"].shape[0], M, prec, torch.cuda.current_stream().cuda_stream, w["kx"], w["ky"])
    sp.spirec_set_data(p.h, w["s"])
    r = w["reg"]
    sp.spirec_set_reg(p.h, r.lambda1, r.alpha1, r.lambda0, r.alpha0, r.kind)
    return p


def _state(sp, p, N):
    G = empty_c64((N, 2 * N - 1))
    D = empty_c64((N, N))
    sp.spirec_gram_dev(p.h, G)
    sp.spirec_data_adjoint_dev(p.h, D)
    return from_dev(G), from_dev(D)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("objective", [0, 1])
def test_autotune_state_equals_a_new_plan(sp, prec, objective):
    w = _workload()
    N, L = w["N"], w["kx"].shape[0]
    with _plan(sp, w, prec, 128) as p:
        chosen, ms = sp.spirec_autotune(p.h, objective, 5)
        tiles = [sp.SPIREC_KNOB_GRAM_TILE, sp.SPIREC_KNOB_ADJOINT_TILE]
        rest = [k for k in range(sp.SPIREC_NUM_KNOBS) if k not in tiles]
        # M = 128: the loop is tuned too; the tile shapes only on the tensor-core paths
        assert np.all(chosen[rest] > 0) and np.all(ms[rest] > 0)
        assert np.all(chosen[tiles] > 0) if prec else np.all(chosen[tiles] == 0)
        for k in range(sp.SPIREC_NUM_KNOBS):
            assert sp.spirec_tune_get(k, N, p.M, prec, L) == chosen[k]
        G1, D1 = _state(sp, p, N)
        x1, J1 = sp.spirec_solve(p.h, None, 12, N)
        M = p.M
    with _plan(sp, w, prec, M) as q:
        G2, D2 = _state(sp, q, N)
        x2, J2 = sp.spirec_solve(q.h, None, 12, N)
    assert np.array_equal(G1, G2) and np.array_equal(D1, D2)
    assert np.array_equal(x1, x2) and np.array_equal(J1, J2)
    xo, Jo, _ = O.solve(w["kx"], w["ky"], w["s"], w["reg"], np.zeros((N, N)), 12)
    assert rel(J1, Jo) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_every_split_matches_the_oracle(sp, prec):
    """G and D under split values from one slice / CTA to more than the
    work has (clipped), against the oracle."""
    w = _workload(N=40, I=2, S=1100, seed=22)
    N, L = w["N"], w["kx"].shape[0]
    Go = O.gram(w["kx"], w["ky"], N)[:, N - 1:].T
    Do = O.adjoint(w["kx"], w["ky"], w["s"], N)
    M = 2 * N
    for v in [1, 2, 3, 7, 19, 50, 152, 1000]:
        sp.spirec_tune_set(sp.SPIREC_KNOB_GRAM_SPLIT, N, M, prec, L, v)
        sp.spirec_tune_set(sp.SPIREC_KNOB_ADJOINT_SPLIT, N, M, prec, L, v)
        with _plan(sp, w, prec, M) as p:
            G, D = _state(sp, p, N)
        assert rel(G, Go) < TOL[prec], v
        assert rel(D, Do) < TOL[prec], v


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("N", [40, 200, 300])
def test_every_tile_shape_matches_the_oracle(sp, prec, N):
    """G and D with one SM a tile (128 rows) and with CTA pairs (256 rows),
    each under a few CTA counts (odd ones rounded down to pairs), against
    sampled oracle entries: N = 40 leaves most of a tile's rows empty, 200
    one ragged tile of either shape, 300 several tiles with ragged edges."""
    w = _workload(N=N, I=2, S=4 * N, seed=29)
    L = w["kx"].shape[0]
    M = 2 * N
    g = synth.rng(30)
    u = g.integers(0, N, 300)
    v = g.integers(-(N - 1), N, 300)
    n = g.integers(0, N, 300)
    m = g.integers(0, N, 300)
    Go = O.gram_at(w["kx"], w["ky"], N, u, v)
    Do = O.adjoint_at(w["kx"], w["ky"], w["s"], N, n, m)
    try:
        for tile in (1, 2):
            sp.spirec_tune_set(sp.SPIREC_KNOB_GRAM_TILE, N, M, prec, L, tile)
            sp.spirec_tune_set(sp.SPIREC_KNOB_ADJOINT_TILE, N, M, prec, L, tile)
            for val in (3, 38, 152):
                sp.spirec_tune_set(sp.SPIREC_KNOB_GRAM_SPLIT, N, M, prec, L, val)
                sp.spirec_tune_set(sp.SPIREC_KNOB_ADJOINT_SPLIT, N, M, prec, L, val)
                with _plan(sp, w, prec, M) as p:
                    G, D = _state(sp, p, N)
                assert rel(G[u, v + N - 1], Go) < TOL[prec], (tile, val)
                assert rel(D[n, m], Do) < TOL[prec], (tile, val)
    finally:
        sp.spirec_tune_clear()


@pytest.mark.parametrize("prec", [1, 2])
def test_fewer_ctas_than_tiles(sp, prec):
    """N = 300: G has 3 x 3 output tiles and D 3 x 2, so CTA counts below
    the tile count give CTAs whose sample ranges span several tiles; sampled
    entries against the oracle."""
    w = _workload(N=300, I=2, S=1000, seed=27)
    N, L = w["N"], w["kx"].shape[0]
    M = 600
    g = synth.rng(28)
    u = g.integers(0, N, 400)
    v = g.integers(-(N - 1), N, 400)
    n = g.integers(0, N, 400)
    m = g.integers(0, N, 400)
    Go = O.gram_at(w["kx"], w["ky"], N, u, v)
    Do = O.adjoint_at(w["kx"], w["ky"], w["s"], N, n, m)
    for val in [1, 2, 5, 8, 152]:
        sp.spirec_tune_set(sp.SPIREC_KNOB_GRAM_SPLIT, N, M, prec, L, val)
        sp.spirec_tune_set(sp.SPIREC_KNOB_ADJOINT_SPLIT, N, M, prec, L, val)
        with _plan(sp, w, prec, M) as p:
            G, D = _state(sp, p, N)
        assert rel(G[u, v + N - 1], Go) < TOL[prec], val
        assert rel(D[n, m], Do) < TOL[prec], val


@pytest.mark.parametrize("N,M", [(48, 128), (100, 256), (260, 1024)])
def test_every_loop_shape_matches_the_oracle(sp, N, M):
    """The persistent loop with each rows-per-block value the tuner tries,
    and odd ones (the last block owns fewer rows), against the oracle; a
    value whose blocks do not fit falls back to the heuristic's shape."""
    w = _workload(N=N, I=3, S=5 * N, seed=23)
    iters = 6
    xo, Jo, _ = O.solve(w["kx"], w["ky"], w["s"], w["reg"], np.zeros((N, N)), iters)
    rpc = 4 * 512 // M
    for rb in [rpc * g for g in range(1, 9) if rpc * (g - 1) < N] + [1, 3, 7]:
        sp.spirec_tune_set(sp.SPIREC_KNOB_LOOP_ROWS, N, M, 0, 1, rb)
        with _plan(sp, w, 0, M) as p:
            x, J = sp.spirec_solve(p.h, None, iters, N)
        assert rel(J, Jo) < 1e-5, rb
        assert rel(x, xo) < 1e-4, rb
    sp.spirec_tune_set(sp.SPIREC_KNOB_LOOP_ROWS, N, M, 0, 1, 100000)  # far beyond shared memory
    with _plan(sp, w, 0, M) as p:
        x_big, _ = sp.spirec_solve(p.h, None, iters, N)
    sp.spirec_tune_clear()
    with _plan(sp, w, 0, M) as p:
        x_def, _ = sp.spirec_solve(p.h, None, iters, N)
    assert np.array_equal(x_big, x_def)


def test_iteration_graph_follows_the_table(sp):
    """Direct mode replays a captured graph of its iterations; after a table
    change the next solve re-captures with the new split."""
    w = _workload(N=32, I=2, S=500, seed=24)
    N, L = w["N"], w["kx"].shape[0]
    M = 64
    with _plan(sp, w, 1, M) as p:
        sp.spirec_set_mode(p.h, sp.SPIREC_MODE_DIRECT)
        sp.spirec_solve(p.h, None, 4, N)
        sp.spirec_tune_set(sp.SPIREC_KNOB_ADJOINT_SPLIT, N, M, 1, L, 3)
        sp.spirec_set_trajectory(p.h, w["kx"], w["ky"])
        sp.spirec_set_data(p.h, w["s"])
        x1, J1 = sp.spirec_solve(p.h, None, 4, N)
    with _plan(sp, w, 1, M) as q:
        sp.spirec_set_mode(q.h, sp.SPIREC_MODE_DIRECT)
        x2, J2 = sp.spirec_solve(q.h, None, 4, N)
    assert np.array_equal(x1, x2) and np.array_equal(J1, J2)


def test_save_load_on_the_device(sp, tmp_path):
    w = _workload(N=32, I=2, S=400, seed=25)
    N, L = w["N"], w["kx"].shape[0]
    with _plan(sp, w, 2) as p:
        chosen, _ = sp.spirec_autotune(p.h, 1, 3)
        M = p.M
    path = str(tmp_path / "t.txt")
    sp.spirec_tune_save(path)
    sp.spirec_tune_clear()
    sp.spirec_tune_load(path)
    for k in range(3):
        assert sp.spirec_tune_get(k, N, M, 2, L) == chosen[k]


def test_autotune_errors(sp):
    w = _workload(N=32, I=2, S=400, seed=26)
    import torch
    with sp.Plan(32, w["kx"].shape[0], 0, 1, torch.cuda.current_stream().cuda_stream, w["kx"], w["ky"]) as p:
        with pytest.raises(sp.SpirecError) as e:  # no data yet
            sp.spirec_autotune(p.h, 0, 3)
        assert e.value.code == sp.SPIREC_ESTATE
        sp.spirec_set_data(p.h, w["s"])
        sp.spirec_set_reg(p.h, 0.05, 0.05, 0.0, 0.05, 0)
        for bad in [(2, 3), (0, 0)]:
            with pytest.raises(sp.SpirecError) as e:
                sp.spirec_autotune(p.h, *bad)
            assert e.value.code == sp.SPIREC_EINVAL
        assert sp.spirec_tune_count() == 0
