"""The per-interleave kernel cache: G (Eq. AnnMatG) sums over the samples and
the kernel spectrum is linear in G, so a plan whose trajectory is set from
cached interleaves must carry the same G and spectrum (to FP32 rounding) as
one built from the concatenated samples, and reach the same solve."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0908_3252_gb300 import synth
from tests.helpers import c64, empty_c64, from_dev, rel

pytestmark = pytest.mark.gpu

N, I, S = 64, 16, 256
WHICH = [3, 7, 11, 14]


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
def series():
    kx, ky = synth.spiral(N, I, S, "archimedean", "golden")
    idx = np.concatenate([np.arange(j * S, (j + 1) * S) for j in WHICH])
    f = synth.phantom(N, "ellipses_phase", synth.rng(61))
    s = c64(synth.add_noise(O.forward(kx[idx], ky[idx], f), 30.0, synth.rng(62)))
    reg = O.Reg(0.05, 0.05, 0.0, 0.05, O.PHI_HUBER)
    xo, Jo, _ = O.solve(kx[idx], ky[idx], s, reg, np.zeros((N, N)), 20)
    return dict(kx=kx, ky=ky, idx=idx, s=s, reg=reg, xo=xo, Jo=Jo)


@pytest.mark.parametrize("prec", [0, 1])
def test_cached_trajectory_equals_built_one(sp, series, prec):
    import torch
    kx, ky, idx = series["kx"], series["ky"], series["idx"]
    offsets = np.arange(0, I * S + 1, S)
    cache = sp.spirec_kcache_create(N, 0, prec, offsets, kx, ky)
    try:
        out = {}
        for mode in ("built", "cached"):
            with sp.Plan(N, idx.shape[0], 0, prec, torch.cuda.current_stream().cuda_stream) as p:
                if mode == "built":
                    sp.spirec_set_trajectory(p.h, kx[idx], ky[idx])
                else:
                    sp.spirec_set_trajectory_cached(p.h, cache, WHICH)
                G = empty_c64((N, 2 * N - 1))
                sp.spirec_gram_dev(p.h, G)
                C = torch.zeros((p.M, p.M), dtype=torch.float32, device="cuda")
                sp.spirec_kernel_spectrum_dev(p.h, C)
                reg = series["reg"]
                sp.spirec_set_data(p.h, series["s"])
                sp.spirec_set_reg(p.h, reg.lambda1, reg.alpha1, reg.lambda0, reg.alpha0, reg.kind)
                x, J = sp.spirec_solve(p.h, None, 20, N)
                out[mode] = (from_dev(G), from_dev(C), x, J)
    finally:
        sp.spirec_kcache_destroy(cache)
    (Gb, Cb, xb, Jb), (Gc, Cc, xc, Jc) = out["built"], out["cached"]
    assert rel(Gc, Gb) < 1e-6
    assert rel(Cc, Cb) < 1e-6
    assert rel(xc, xb) < 1e-4
    for x, J in ((xb, Jb), (xc, Jc)):
        assert rel(J, series["Jo"]) < (1e-5 if prec == 0 else 1e-3)
        assert rel(x, series["xo"]) < 1e-3


def test_cache_argument_errors(sp, series):
    kx, ky = series["kx"], series["ky"]
    offsets = np.arange(0, I * S + 1, S)
    with pytest.raises(sp.SpirecError) as e:
        sp.spirec_kcache_create(N, 0, 0, np.array([0, 10, 10]), kx, ky)
    assert e.value.code == sp.SPIREC_EINVAL
    cache = sp.spirec_kcache_create(N, 0, 0, offsets, kx, ky)
    try:
        with sp.Plan(N, 4 * S, 0, 0) as p:
            for bad in ([3, 7, 11], [3, 7, 11, 16], [3, 7, 11, -1]):
                with pytest.raises(sp.SpirecError) as e:
                    sp.spirec_set_trajectory_cached(p.h, cache, bad)
                assert e.value.code == sp.SPIREC_EINVAL
        with sp.Plan(N + 2, 4 * S, 0, 0) as p:
            with pytest.raises(sp.SpirecError) as e:
                sp.spirec_set_trajectory_cached(p.h, cache, WHICH)
            assert e.value.code == sp.SPIREC_EINVAL
    finally:
        sp.spirec_kcache_destroy(cache)


@pytest.mark.parametrize("prec", [0, 1])
def test_captured_series_matches_the_oracle(sp, prec):
    """A dynamic series as the benchmark runs it, small: six frames of sizes
    32, 48 and 64, each using 4 of 16 golden-angle interleaves from a kernel
    cache, each with its own plan and stream; every frame's trajectory (from
    the cache), data and 20 iterations are captured as ONE CUDA graph (fork
    from a capture stream, join back) and replayed twice.  Every frame of
    the replays is compared with the oracle's 20 iterations on the frame's
    own samples, and the two replays with each other (bitwise)."""
    import torch
    from tests.helpers import iter_tol
    g = synth.rng(71)
    S16 = 256
    kx16, ky16 = synth.spiral(64, 16, S16, "archimedean", "golden")
    offsets = np.arange(0, 16 * S16 + 1, S16)
    Ms = {32: 64, 48: 128, 64: 128}
    caches = {n: sp.spirec_kcache_create(n, m, prec, offsets, kx16, ky16) for n, m in Ms.items()}
    frames, keep = [], []
    iters = 20
    try:
        for i, n in enumerate([32, 48, 64, 48, 32, 64]):
            sub = np.sort(g.choice(16, 4, replace=False)).astype(np.int32)
            idx = np.concatenate([np.arange(j * S16, (j + 1) * S16) for j in sub])
            kx, ky = kx16[idx], ky16[idx]
            f = synth.phantom(n, "ellipses_phase", synth.rng(80 + i))
            s = c64(synth.add_noise(O.forward(kx, ky, f), 30.0, g))
            st = torch.cuda.Stream()
            p = sp.Plan(n, kx.shape[0], Ms[n], prec, st.cuda_stream)
            s_d = torch.from_numpy(s.astype(np.complex64)).cuda()
            x = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
            sp.spirec_set_reg(p.h, 0.05, 0.05, 0.0, 0.05, 0)
            frames.append(dict(p=p, st=st, s_d=s_d, x=x, sub=sub, kx=kx, ky=ky, s=s, N=n, cache=caches[n]))
        torch.cuda.synchronize()

        def frame(fr):
            sp.spirec_set_trajectory_cached(fr["p"].h, fr["cache"], fr["sub"])
            sp.spirec_set_data_dev(fr["p"].h, fr["s_d"])
            sp.spirec_solve_dev(fr["p"].h, None, iters, fr["x"], None)

        for fr in frames:  # every plan's buffers and kernels in place before capture
            frame(fr)
        torch.cuda.synchronize()
        cap = torch.cuda.Stream()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=cap):
            fork = torch.cuda.Event()
            fork.record(cap)
            joins = []
            for fr in frames:
                fr["st"].wait_event(fork)
                frame(fr)
                e = torch.cuda.Event()
                e.record(fr["st"])
                joins.append(e)
            for e in joins:
                cap.wait_event(e)
        results = []
        for _ in range(2):
            for fr in frames:
                fr["x"].zero_()
            torch.cuda.synchronize()
            graph.replay()
            torch.cuda.synchronize()
            results.append([fr["x"].cpu().numpy() for fr in frames])
        for fr in frames:
            sp.spirec_sync(fr["p"].h)
        del graph
    finally:
        for fr in frames:
            fr["p"].close()
        for c in caches.values():
            sp.spirec_kcache_destroy(c)
    reg = O.Reg(0.05, 0.05, 0.0, 0.05, O.PHI_HUBER)
    for fr, x1, x2 in zip(frames, results[0], results[1]):
        assert np.array_equal(x1, x2)
        n = fr["N"]
        xo, _, _ = O.solve(fr["kx"], fr["ky"], fr["s"], reg, np.zeros((n, n)), iters)
        w = dict(N=n, kx=fr["kx"], ky=fr["ky"], s=fr["s"], reg=reg, iters=iters)
        assert rel(x1, xo) < max(1e-3, iter_tol(w, prec)), (n, rel(x1, xo))
