#!/usr/bin/env python3
"""Benchmark: CG iterations/s of a full 512x512 regularized spiral
reconstruction on GB300 (one JSON line on stdout).

One step = the whole hot path on one synthetic acquisition, through the C ABI
with inputs already resident in HBM:
    set_trajectory_dev  (fixed-point trajectory, G build, kernel spectrum)
    set_data_dev        (||s||^2, D = H^H s)
    solve_dev           (50 Polak-Ribiere CG iterations on the Toeplitz form)
value = 50 * steps / (sum of per-step device times); the L2 cache is flushed
(256 MB write) before every timed step.  e2e repeats the step through the
host-pointer API (pinned host buffers, copies inside the timed region).

Workload (512x512, the metric's configuration): ellipses x smooth complex
phase + 40 bars + texture, Archimedean spiral 32 x 4096 (L = 131072), 30 dB
noise, Huber phi alpha 0.05, lambda 0.05, M = 1024, 50 iterations, seed 3.

--impl reference times the FP64 CPU oracle (direct NUDFT form of the same
minimiser) on a bounded sample of the same workload, on the host cores.
Under torchrun every rank runs its own reconstructions (replicas; the
reconstructions are independent), value = all ranks' iterations / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CG iters/s at 512^2 (mixed-prec vs FP32 plain, <=1e-3 err); p50/p99 latency"
UNIT = "iters/s"
ITERS = 50
# DRAM bytes (read + write) per launch of the dominant kernels on the default
# workload: dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture
# (--clock-control none) of the persistent CG loop over 50 iterations and of
# one G and one D contraction, each with the digest of the sources the kernel
# is built from at the time of the capture.  A figure whose sources have
# changed since is reported as null: the counters no longer describe the
# kernel that runs.
NCU_TRAFFIC = {"k_cg_loop": (10_712_832, "9a5d48a08d744779"), "k_tc_pair_gemm_G": (2_171_904, "09eacbd42c77e41e"),
               "k_tc_pair_gemm_D": (3_207_936, "09eacbd42c77e41e")}
KERNEL_SOURCES = {
    "k_cg_loop": ["cg_loop.cu", "cg_device.cuh", "fft_device.cuh", "fft_reg.cuh", "reduce.cuh", "penalty.cuh",
                  "internal.cuh"],
    "k_tc_pair_gemm_G": ["nudft_tc.cu", "phase.cuh", "internal.cuh"],
    "k_tc_pair_gemm_D": ["nudft_tc.cu", "phase.cuh", "internal.cuh"],
}


def source_digest(kernel):
    """16 hex digits of the SHA-256 of the kernel's source files, in order."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_0908_3252_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """The captured DRAM bytes of the kernel if its sources are unchanged, else None."""
    nbytes, digest = NCU_TRAFFIC.get(kernel, (None, None))
    return nbytes if nbytes is not None and digest == source_digest(kernel) else None


def workload(seed=3, S=4096):
    from paper_0908_3252_gb300 import synth
    N, I = 512, 32
    g = synth.rng(seed)
    f_true = synth.phantom(N, "edges_texture", g)
    kx, ky = synth.spiral(N, I, S, "archimedean")
    return dict(N=N, M=1024, kx=kx, ky=ky, f_true=f_true, g=g, snr=30.0,
                lambda1=0.05, alpha1=0.05, lambda0=0.0, alpha0=0.05, phi=0,
                name=f"512x512 edges+texture phantom, Archimedean spiral {I}x{S} (L={I * S}), "
                     f"30 dB, Huber a=0.05 l=0.05, M=1024, {ITERS} CG iters")


def apply_size_args(args):
    """--samples / --iters shrink the workload for profiling captures only;
    the default is the metric's configuration."""
    global ITERS
    ITERS = args.iters


def run_batch(spirec, prec, frames=64, iters=50, seed=4):
    """Dynamic series: `frames` frames, sizes from {128, 192, 256}, each
    sampling 4 of 16 golden-angle interleaves x 2048 (L = 8192), moving
    ellipse phantoms; every frame's trajectory, data and solve on its own
    plan's stream, the whole series captured as one CUDA graph and timed as
    one replay.  Launch shapes are autotuned for throughput (one frame per
    image size; the heuristic shapes are timed too).  Timed twice: with each frame's G and spectrum built from its
    samples, and set from a per-interleave kernel cache (the spectrum of a
    subset is the sum of its interleaves' spectra; the cache is built once
    per image size, outside the timed region, and its build time reported)."""
    import torch
    from paper_0908_3252_gb300 import synth
    g = synth.rng(seed)
    kx16, ky16 = synth.spiral(256, 16, 2048, "archimedean", "golden")
    offsets = np.arange(0, 16 * 2048 + 1, 2048)
    Ms = {128: 256, 192: 512, 256: 512}
    t0 = time.perf_counter()
    caches = {N: spirec.spirec_kcache_create(N, M, prec, offsets, kx16, ky16) for N, M in Ms.items()}
    cache_s = time.perf_counter() - t0
    items = []
    for i in range(frames):
        N = int(g.choice([128, 192, 256]))
        sub = np.sort(g.choice(16, 4, replace=False))
        idx = np.concatenate([np.arange(j * 2048, (j + 1) * 2048) for j in sub])
        kx, ky = kx16[idx], ky16[idx]
        L = kx.shape[0]
        f = synth.ellipses(N, 10, synth.rng(1000 + i)).astype(np.complex64)
        st = torch.cuda.Stream()
        p = spirec.Plan(N, L, Ms[N], prec, st.cuda_stream)
        kx_d, ky_d = torch.from_numpy(kx).cuda(), torch.from_numpy(ky).cuda()
        torch.cuda.synchronize()
        spirec.spirec_set_trajectory_dev(p.h, kx_d, ky_d)
        y = torch.zeros(L, dtype=torch.complex64, device="cuda")
        spirec.spirec_forward_dev(p.h, torch.from_numpy(f).cuda(), y)
        spirec.spirec_sync(p.h)
        s_d = torch.from_numpy(synth.add_noise(y.cpu().numpy().astype(np.complex128), 30.0, g)
                               .astype(np.complex64)).cuda()
        spirec.spirec_set_reg(p.h, 0.05, 0.05, 0.0, 0.05, 0)
        x = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
        items.append((p, st, kx_d, ky_d, s_d, x, caches[N], sub.astype(np.int32)))

    def frame(it, cached):
        p, st, kx_d, ky_d, s_d, x, cache, sub = it
        if cached:
            spirec.spirec_set_trajectory_cached(p.h, cache, sub)
        else:
            spirec.spirec_set_trajectory_dev(p.h, kx_d, ky_d)
        spirec.spirec_set_data_dev(p.h, s_d)
        spirec.spirec_solve_dev(p.h, None, iters, x, None)

    def timed_graph(cached):
        for it in items:  # warm-up: every plan's buffers and kernels are in place
            frame(it, cached)
        torch.cuda.synchronize()
        # the whole series as ONE CUDA graph: fork from a capture stream to
        # every frame's stream, each frame's trajectory, data and solve, join
        cap = torch.cuda.Stream()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=cap):
            fork = torch.cuda.Event()
            fork.record(cap)
            joins = []
            for it in items:
                it[1].wait_event(fork)
                frame(it, cached)
                e = torch.cuda.Event()
                e.record(it[1])
                joins.append(e)
            for e in joins:
                cap.wait_event(e)
        graph.replay()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(cap)
        graph.replay()
        e1.record(cap)
        torch.cuda.synchronize()
        del graph
        return e0.elapsed_time(e1) / 1000.0

    # autotune one frame plan per image size for throughput (the frames share
    # the GPU); every frame of that size then launches with the chosen splits
    # and loop shape.  The series is also timed with the built-in heuristics.
    spirec.spirec_tune_clear()
    dt_default = timed_graph(True)
    t0 = time.perf_counter()
    tuned = {}
    for N in sorted(Ms):
        it = next((it for it in items if it[0].N == N), None)
        if it is None:
            continue
        p = it[0]
        spirec.spirec_set_data_dev(p.h, it[4])
        chosen, _ = spirec.spirec_autotune(p.h, spirec.SPIREC_TUNE_THROUGHPUT, iters)
        tuned[N] = dict(zip(("gram_split", "adjoint_split", "loop_rows", "gram_tile", "adjoint_tile"),
                            chosen.tolist()))
    tune_s = time.perf_counter() - t0
    dt_built = timed_graph(False)
    dt = timed_graph(True)
    spirec.spirec_tune_clear()
    sizes = sorted({it[0].N for it in items})
    for it in items:
        it[0].close()
    for c in caches.values():
        spirec.spirec_kcache_destroy(c)
    return {"frames": frames, "sizes": sizes, "iters": iters, "seconds": dt,
            "frames_per_s": frames / dt, "iters_per_s": frames * iters / dt,
            "frames_per_s_built_G": frames / dt_built, "kernel_cache_build_s": cache_s,
            "frames_per_s_heuristic_shapes": frames / dt_default, "autotuned": tuned, "autotune_s": tune_s,
            "what": "per frame: trajectory (spectrum from the kernel cache), data (D), 50 CG iterations; "
                    "the 64 frames on their own streams, captured as one CUDA graph and timed as one replay"}


def run_paper_experiment(spirec, prec, iters=50, reps=20):
    """The paper's simulated experiment (section 4.1) with a stand-in for its
    phantom: 128 x 128 two-vessel image (intensity ~255), 6 spiral arms x 512
    samples, 30 dB, Huber phi with lambda1 = 0.1, alpha1 = 20, lambda0 = 0.5,
    alpha0 = 10, 50 iterations.  The paper's figures of merit (quadratic
    error in ROI1, variance in ROI2) for that reconstruction and for the
    unregularized one, and the solve rate (trajectory, data and 50
    iterations per reconstruction)."""
    import torch
    from paper_0908_3252_gb300 import synth
    N = 128
    f, roi = synth.vessels(N)
    kx, ky = synth.spiral(N, 6, 512, "archimedean")
    L = kx.shape[0]
    st = torch.cuda.Stream()
    p = spirec.Plan(N, L, 0, prec, st.cuda_stream)
    kx_d, ky_d = torch.from_numpy(kx).cuda(), torch.from_numpy(ky).cuda()
    torch.cuda.synchronize()
    spirec.spirec_set_trajectory_dev(p.h, kx_d, ky_d)
    y = torch.zeros(L, dtype=torch.complex64, device="cuda")
    spirec.spirec_forward_dev(p.h, torch.from_numpy(f.astype(np.complex64)).cuda(), y)
    spirec.spirec_sync(p.h)
    s_d = torch.from_numpy(synth.add_noise(y.cpu().numpy().astype(np.complex128), 30.0, synth.rng(51))
                           .astype(np.complex64)).cuda()
    x = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
    J = torch.zeros(iters + 1, dtype=torch.float64, device="cuda")
    out = {"N": N, "samples": L, "iters": iters}
    for name, reg in (("regularized", (0.1, 20.0, 0.5, 10.0, 0)), ("unregularized", (0.0, 20.0, 0.0, 10.0, 0))):
        spirec.spirec_set_reg(p.h, *reg)
        with torch.cuda.stream(st):
            spirec.spirec_set_data_dev(p.h, s_d)
            spirec.spirec_solve_dev(p.h, None, iters, x, J)
        torch.cuda.synchronize()
        xr = x.cpu().numpy().astype(np.complex128)
        err = float(np.sum(np.abs(xr - f)[roi["roi1"]] ** 2) / np.sum(np.abs(f)[roi["roi1"]] ** 2))
        out[name] = {"roi1_quadratic_error": err, "roi2_variance": float(np.var(np.abs(xr)[roi["roi2"]]))}
    spirec.spirec_set_reg(p.h, 0.1, 20.0, 0.5, 10.0, 0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        spirec.spirec_set_trajectory_dev(p.h, kx_d, ky_d)
        spirec.spirec_set_data_dev(p.h, s_d)
        spirec.spirec_solve_dev(p.h, None, iters, x, J)
    e1.record(st)
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) / 1000.0 / reps
    p.close()
    out["ms_per_reconstruction"] = dt * 1e3
    out["iters_per_s"] = iters / dt
    return out


def run_direct_mode(spirec, prec, w, s_host):
    """The paper's claim for its rewriting (section 3.4): the cost of one CG
    iteration when H^H H is applied by the Toeplitz FFT convolution against
    the original formulation, which applies the exact forward and adjoint
    NUDFT every iteration (SPIREC_MODE_DIRECT).  Steady state, per
    iteration: (time of a 10-iteration solve - time of a 2-iteration solve) / 8,
    on the metric's 512^2 workload with G, Chat and D in place."""
    import torch
    N, M, L = w["N"], w["M"], w["kx"].shape[0]
    st = torch.cuda.Stream()
    p = spirec.Plan(N, L, M, prec, st.cuda_stream, w["kx"], w["ky"])
    spirec.spirec_set_data(p.h, s_host)
    spirec.spirec_set_reg(p.h, w["lambda1"], w["alpha1"], w["lambda0"], w["alpha0"], w["phi"])
    x = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
    out = {}
    for name, mode in (("toeplitz", spirec.SPIREC_MODE_TOEPLITZ), ("direct", spirec.SPIREC_MODE_DIRECT)):
        spirec.spirec_set_mode(p.h, mode)
        t = {}
        for iters in (2, 10, 2, 10):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            spirec.spirec_solve_dev(p.h, None, iters, x, None)
            e1.record(st)
            torch.cuda.synchronize()
            t[iters] = e0.elapsed_time(e1)  # the second (warm) run of each count stays
        out[name + "_ms_per_iter"] = (t[10] - t[2]) / 8.0
    p.close()
    out["rewriting_speedup"] = out["direct_ms_per_iter"] / out["toeplitz_ms_per_iter"]
    return out


def run_half_quadratic(spirec, prec, w, s_host, budget=50, ref_iters=400):
    """The two replacements for the conjugate gradient that section 5 names,
    the half-quadratic (dual) minimiser and the truncated Newton one, against
    PR+ CG at an equal budget of T applies on the metric's 512^2 workload:
    PR+ CG for `budget` iterations, the others for outer x inner = budget.
    Reports each run's final J, its gap to J* (PR+ CG after ref_iters
    iterations, relative to J(0) - J*) and its time (events on the plan's
    stream, second of two runs)."""
    import torch
    N, M, L = w["N"], w["M"], w["kx"].shape[0]
    st = torch.cuda.Stream()
    p = spirec.Plan(N, L, M, prec, st.cuda_stream, w["kx"], w["ky"])
    spirec.spirec_set_data(p.h, s_host)
    spirec.spirec_set_reg(p.h, w["lambda1"], w["alpha1"], w["lambda0"], w["alpha0"], w["phi"])
    x = torch.zeros((N, N), dtype=torch.complex64, device="cuda")

    def run(kind, inner, iters):
        spirec.spirec_set_minimiser(p.h, kind, inner)
        J = torch.zeros(iters + 1, dtype=torch.float64, device="cuda")
        ms = 0.0
        for _ in range(2):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            spirec.spirec_solve_dev(p.h, None, iters, x, J)
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
        return J.cpu().numpy(), ms

    Jref, _ = run(spirec.SPIREC_MIN_PRCG, 0, ref_iters)
    J0, Jstar = float(Jref[0]), float(Jref[-1])
    out = {"budget_T_applies": budget, "J0": J0, "J_star_prcg_%d" % ref_iters: Jstar, "runs": {}}

    def entry(J, ms):
        return {"J": float(J[-1]), "gap": (float(J[-1]) - Jstar) / (J0 - Jstar), "ms": ms}

    J, ms = run(spirec.SPIREC_MIN_PRCG, 0, budget)
    out["runs"]["prcg_%d" % budget] = entry(J, ms)
    for inner in (2, 5, 10):
        J, ms = run(spirec.SPIREC_MIN_HALF_QUADRATIC, inner, budget // inner)
        out["runs"]["hq_%dx%d" % (budget // inner, inner)] = entry(J, ms)
    for inner in (5, 10, 25):
        J, ms = run(spirec.SPIREC_MIN_NEWTON, inner, budget // inner)
        out["runs"]["newton_%dx%d" % (budget // inner, inner)] = entry(J, ms)
    p.close()
    return out


def run_graph_path(spirec, prec, N=2048, M=4096, interleaves=64, samples=2048, hbm_gbs=None):
    """The CG iteration as separate kernels in a captured graph (row FFTs with
    the fused direction and first line-search sums, column filter, row IFFTs
    with q2, two line-search steps, update), on an image whose working set
    (about 320 MB: f, d, g, T f, T d, D, the N x M rows, the spectrum) is far
    beyond the 129 MB L2, so that these FFT and stencil kernels stream through
    HBM: 2048 x 2048, M = 4096 (beyond the persistent loop's sizes), spiral
    64 x 2048 (L = 131072).  Steady-state time per iteration from solves of 2
    and 12 iterations (events, second of two runs), and the algorithmic bytes
    per iteration (160 N^2) over it."""
    import torch
    from paper_0908_3252_gb300 import synth
    g = synth.rng(7)
    kx, ky = synth.spiral(N, interleaves, samples, "archimedean")
    L = kx.shape[0]
    f = synth.ellipses(N, 10, g).astype(np.complex64)
    st = torch.cuda.Stream()
    p = spirec.Plan(N, L, M, prec, st.cuda_stream, kx, ky)
    y = torch.zeros(L, dtype=torch.complex64, device="cuda")
    spirec.spirec_forward_dev(p.h, torch.from_numpy(f).cuda(), y)
    spirec.spirec_set_data_dev(p.h, y)
    spirec.spirec_set_reg(p.h, 0.05, 0.05, 0.0, 0.05, 0)
    x = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
    t = {}
    for iters in (2, 12, 2, 12):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        spirec.spirec_solve_dev(p.h, None, iters, x, None)
        e1.record(st)
        torch.cuda.synchronize()
        t[iters] = e0.elapsed_time(e1)
    p.close()
    ms = (t[12] - t[2]) / 10.0
    gbs = 160.0 * N * N / (ms / 1e3) / 1e9
    out = {"N": N, "M": M, "L": L, "ms_per_iter": ms, "algorithmic_bytes_per_iter": 160 * N * N,
           "algorithmic_GBps": gbs,
           "path": "stand-alone kernels in a captured graph (M = 4096 is beyond the persistent loop)"}
    if hbm_gbs:
        out["frac_of_measured_hbm"] = gbs / hbm_gbs
    return out


def run_serving(spirec, prec, requests=2000, rate=200.0, iters=50, seed=5, slots=8):
    """Poisson request stream: sizes N in {64..384} step 64, L uniform in
    [8000, 200000] (spiral of ceil(L/2048) interleaves truncated to L),
    lambda1 U[0.01, 0.2], Huber alpha 0.05, 50 iterations; p50/p99 latency
    from submission to result, and requests/s over the whole stream."""
    from paper_0908_3252_gb300 import synth
    g = synth.rng(seed)
    reqs = []
    for _ in range(requests):
        N = int(g.choice(np.arange(64, 385, 64)))
        L = int(g.integers(8000, 200001))
        I = (L + 2047) // 2048
        kx, ky = synth.spiral(N, I, 2048)
        kx, ky = kx[:L].copy(), ky[:L].copy()
        s = synth.complex_normal(L, g).astype(np.complex64)
        reqs.append((N, kx, ky, s, float(g.uniform(0.01, 0.2))))
    gaps = g.exponential(1.0 / rate, requests)
    srv = spirec.spirec_server_create(64 << 30, slots, prec)
    try:
        t0 = time.perf_counter()
        next_t = t0
        tickets = []
        for (N, kx, ky, s, lam), gap in zip(reqs, gaps):
            next_t += gap
            delay = next_t - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append((spirec.spirec_server_submit(srv, N, kx, ky, s, lam, 0.05, 0.0, 0.05, 0, iters), N))
        for t, N in tickets:
            spirec.spirec_server_wait(srv, t, N, timeout_ms=600000)
        dt = time.perf_counter() - t0
        st = spirec.spirec_server_stats(srv)
    finally:
        spirec.spirec_server_destroy(srv)
    return {"requests": requests, "arrival_rate_per_s": rate, "slots": slots, "p50_ms": st["p50_s"] * 1e3,
            "p99_ms": st["p99_s"] * 1e3, "requests_per_s": requests / dt, "failed": st["failed"]}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# Clock-event reason bits of NVML (nvmlClocksEventReason*).
_NVML_REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
                 0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}


class _NvmlClocks:
    """SM clock and clock-event reasons of this process's GPU, read through
    NVML every millisecond or so by a host thread while the timed region runs
    (read-only queries; nothing is set).  The GPU is matched by PCI bus id."""

    def __init__(self, device):
        import ctypes
        import threading
        import torch
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        pr = torch.cuda.get_device_properties(device)
        self.h = ctypes.c_void_p()
        bus = getattr(pr, "pci_bus_id", None)
        rc = -1
        if bus is not None:
            pci = "%08X:%02X:%02X.0" % (getattr(pr, "pci_domain_id", 0), bus, getattr(pr, "pci_device_id", 0))
            rc = self.lib.nvmlDeviceGetHandleByPciBusId_v2(pci.encode(), ctypes.byref(self.h))
        if rc != 0 and self.lib.nvmlDeviceGetHandleByIndex_v2(device, ctypes.byref(self.h)) != 0:
            raise OSError("no NVML handle")
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint()
        self.max_mhz = float(mx.value) if self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0 \
            else None
        self.samples = []
        self.stop_ev = threading.Event()
        self.thread = threading.Thread(target=self._run, daemon=True)
        self.ctypes = ctypes

    def _run(self):
        ct = self.ctypes
        mhz, rs = ct.c_uint(), ct.c_ulonglong()
        while not self.stop_ev.is_set():
            if self.lib.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(mhz)) == 0 and \
                    self.reasons_fn(self.h, ct.byref(rs)) == 0:
                self.samples.append((time.time(), float(mhz.value), int(rs.value)))
            time.sleep(0.001)

    def start(self):
        self.thread.start()
        while not self.samples and self.thread.is_alive():  # running before the region starts
            time.sleep(0.001)

    def stop(self):
        self.stop_ev.set()
        self.thread.join(timeout=5)
        self.lib.nvmlShutdown()


def clocks_start(device=0):
    """Starts the clock record of the timed region: the NVML sampler when the
    library loads, else nvidia-smi at its 200 ms period.  The raw samples go
    to clocks_<pid>.csv in the directory named by BENCH_CLOCKS_DIR, when it is
    set and exists; the JSON line carries their summary either way."""
    out_dir = os.environ.get("BENCH_CLOCKS_DIR", "")
    try:
        f = open(os.path.join(out_dir, f"clocks_{os.getpid()}.csv") if out_dir and os.path.isdir(out_dir)
                 else os.devnull, "w")
    except OSError:
        f = open(os.devnull, "w")
    try:
        nv = _NvmlClocks(device)
        nv.start()
        return nv, f
    except Exception:
        pass
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return None, f
    return proc, f


def clocks_stop(proc, f, gpu_index):
    if proc is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    if isinstance(proc, _NvmlClocks):
        proc.stop()
        smp = proc.samples
        f.write("unix_time,sm_mhz,reasons_mask\n")
        for t, m, r in smp:
            f.write(f"{t:.4f},{m:.0f},{r:#x}\n")
        f.close()
        if not smp:
            return {"sm_mhz": None, "sm_max_mhz": proc.max_mhz, "reasons": ["no samples"]}
        reasons = sorted({nm for _, _, r in smp for bit, nm in _NVML_REASONS.items() if r & bit})
        return {"sm_mhz": statistics.median(m for _, m, _ in smp), "sm_max_mhz": proc.max_mhz,
                "sm_min_mhz": min(m for _, m, _ in smp), "samples": len(smp), "reasons": reasons,
                "source": "NVML, sampled every ~1 ms during the timed region"}
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
        out, _ = proc.communicate()
    f.write(out)
    f.close()
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            if int(parts[0]) != gpu_index:
                continue
            sm.append(float(parts[1]))
            smax.append(float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
            "reasons": sorted(reasons), "source": "nvidia-smi -lms 200"}


def job_throughput(local_seconds, units_per_rank, device="cpu"):
    """Whole-job throughput of independent replicas: every rank's units over
    the slowest rank's time (max over ranks through torch.distributed when it
    is initialised, any backend).  Returns (value, max_seconds)."""
    import torch
    import torch.distributed as dist
    t, ws = float(local_seconds), 1
    if dist.is_available() and dist.is_initialized():
        ws = dist.get_world_size()
        tt = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return ws * units_per_rank / t, t


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


# ------------------------------------------------------------ CPU oracle leg

def oracle_sample(w, budget_s=12.0):
    """Times the FP64 oracle's NUDFTs on a bounded sample of the workload and
    extrapolates its CG iterations/s: the oracle minimiser does, per
    iteration, two forward products (H d, H f) and one adjoint (the gradient),
    each N^2 L phase terms; plus one forward and one adjoint to start."""
    from oracle import oracle as O
    N, L = w["N"], w["kx"].shape[0]
    f = w["f_true"]
    rs = np.random.default_rng(0)
    r = (rs.standard_normal(L) + 1j * rs.standard_normal(L))

    def t_forward(ls):
        idx = np.linspace(0, L - 1, ls).astype(np.int64)
        t0 = time.perf_counter()
        O.forward(w["kx"][idx], w["ky"][idx], f)
        return (time.perf_counter() - t0) * L / ls

    def t_adjoint(ps):
        pix = rs.integers(0, N * N, ps)
        t0 = time.perf_counter()
        O.adjoint_at(w["kx"], w["ky"], r, N, (pix // N).astype(np.int32), (pix % N).astype(np.int32))
        return (time.perf_counter() - t0) * (N * N) / ps

    cores = O.num_threads()
    # calibrate on a tiny sample, then size each leg to ~budget/2
    tf = t_forward(cores)
    ta = t_adjoint(cores)
    ls = int(max(cores, min(L, (budget_s / 2) / max(tf / L, 1e-12))))
    ps = int(max(cores, min(N * N, (budget_s / 2) / max(ta / (N * N), 1e-12))))
    TF = t_forward(ls)
    TA = t_adjoint(ps)
    total = ITERS * (2 * TF + TA) + (TF + TA)
    return dict(value=ITERS / total, unit=UNIT, cores=cores, kind="oracle",
                sample=f"oracle FP64 direct NUDFT: forward on {ls} of {L} samples and adjoint on "
                       f"{ps} of {N * N} pixels, extrapolated to {ITERS} iterations "
                       f"(2 forward + 1 adjoint per iteration, +1 of each to start): "
                       f"{total:.3e} s per reconstruction")


def cpu_fp64_leg(spirec, w, dev, model_noise=3e-7):
    """The CPU leg at full size, and every GPU path's error against it.

    The workload's data are simulated by the FP64 forward model (the phantom,
    trajectory and noise draw of the GPU leg); the paper's method then runs on
    the host cores in FP64, timed in full: G (Eq. AnnMatG) and D (Eq.
    AnnMatGD) as matrix products of phase matrices (oracle/factored.py), the
    kernel spectrum, and the 50 iterations of the rewritten criterion with
    zero-padded scipy FFTs (oracle/toeplitz_cpu.py).  On the same data each
    precision's GPU solve is compared with that FP64 solve (iterate relative
    L2, J history on the scale of ||s||^2, final J); beside them stand two
    controls: the FP32 rounding model of the minimiser (oracle/fp32_model.py,
    operator perturbations `model_noise`, the size of the FP32 path's measured
    operator errors) and the FP64 solve with the trajectory moved by 1e-7
    (relative, seeded)."""
    import torch
    from oracle import factored as F
    from oracle import fp32_model as FM
    from oracle import oracle as O
    from oracle import toeplitz_cpu as TC
    from paper_0908_3252_gb300 import synth
    w2 = workload(seed=3, S=w["kx"].shape[0] // 32)
    N, M = w2["N"], w2["M"]
    kx, ky = w2["kx"], w2["ky"]
    L = kx.shape[0]
    s64 = synth.add_noise(F.forward(kx, ky, w2["f_true"]), w2["snr"], w2["g"]).astype(np.complex64)
    reg = O.Reg(w2["lambda1"], w2["alpha1"], w2["lambda0"], w2["alpha0"], w2["phi"])
    x0 = np.zeros((N, N))
    t0 = time.perf_counter()
    G = F.gram(kx, ky, N)
    t_g = time.perf_counter() - t0
    t0 = time.perf_counter()
    D = F.adjoint(kx, ky, s64, N)
    t_d = time.perf_counter() - t0
    t0 = time.perf_counter()
    C = TC.kernel_spectrum(G, N, M)
    ss = float(np.sum(np.abs(s64.astype(np.complex128)) ** 2))
    x64, J64 = TC.solve(C, D, ss, reg, x0, ITERS)
    t_it = time.perf_counter() - t0
    total = t_g + t_d + t_it
    cpu = dict(value=ITERS / total, unit=UNIT, cores=TC.WORKERS,
               kind="the paper's method on the CPU (rewritten criterion, FP64, scipy.fft; G and D as "
                    "FP64 matrix products)",
               seconds={"G": t_g, "D": t_d, "spectrum_and_iterations": t_it},
               sample=f"the full workload ({N}^2, L = {L}, M = {M}, {ITERS} iterations), timed in full")

    def gap(x):
        return float(np.linalg.norm(x - x64) / np.linalg.norm(x64))

    err = {"reference": "FP64 rewritten-criterion solve of the same data (G, D by FP64 matrix products)",
           "data": "the workload's phantom, trajectory and noise draw, simulated by the FP64 forward model"}
    stream = torch.cuda.Stream(device=dev)
    names = {"fp32": spirec.SPIREC_FP32, "fp16x3": spirec.SPIREC_MIXED_FP16X3, "bf16x3": spirec.SPIREC_MIXED_BF16X3}
    for name, prec in names.items():
        p = spirec.Plan(N, L, M, prec, stream.cuda_stream, kx, ky)
        spirec.spirec_set_data(p.h, s64)
        spirec.spirec_set_reg(p.h, w2["lambda1"], w2["alpha1"], w2["lambda0"], w2["alpha0"], w2["phi"])
        x, J = spirec.spirec_solve(p.h, None, ITERS, N)
        p.close()
        x = x.astype(np.complex128)
        err[name] = {"iterate_rel_l2": gap(x), "J_history_max_over_s2": float(np.max(np.abs(J - J64)) / ss),
                     "final_J_rel": float(abs(J[-1] - J64[-1]) / J64[-1]),
                     "error_to_phantom": float(np.linalg.norm(x - w2["f_true"]) / np.linalg.norm(w2["f_true"]))}
    xd, jd = FM.deviations(C, D, ss, reg, x0, ITERS, x64, J64, noise=model_noise, seeds=[0, 1])
    err["fp32_rounding_model"] = {"iterate_rel_l2": xd, "J_history_max_over_s2": [v / ss for v in jd],
                                  "runs": "unperturbed, then seeds 0 and 1", "operator_noise": model_noise}
    pert = 1e-7 * np.random.default_rng(17).standard_normal(L)
    kxp, kyp = kx * (1 + pert), ky * (1 - pert)
    Cp = TC.kernel_spectrum(F.gram(kxp, kyp, N), N, M)
    xp, _ = TC.solve(Cp, F.adjoint(kxp, kyp, s64, N), ss, reg, x0, ITERS)
    err["fp64_k_perturbed_1e-7"] = {"iterate_rel_l2": gap(xp)}
    err["fp64_error_to_phantom"] = float(np.linalg.norm(x64 - w2["f_true"]) / np.linalg.norm(w2["f_true"]))
    return cpu, err


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    w = workload(S=args.samples)
    vals = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample(w, budget_s=3.0)
        if i >= args.warmup:
            vals.append(r["value"])
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * ITERS / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w["name"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ GPU leg

def run_ours(args):
    import torch
    from paper_0908_3252_gb300 import build, spirec, synth
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0:
        build.build()
    if ws > 1:
        dist.barrier()
    spirec.load()

    prec = {"fp32": spirec.SPIREC_FP32, "fp16x3": spirec.SPIREC_MIXED_FP16X3,
            "bf16x3": spirec.SPIREC_MIXED_BF16X3}[args.precision]
    w = workload(seed=3 + rank, S=args.samples)
    N, M = w["N"], w["M"]
    L = w["kx"].shape[0]
    stream = torch.cuda.Stream(device=dev)
    h = spirec.spirec_plan_create(N, L, M, prec, stream.cuda_stream)

    with torch.cuda.stream(stream):
        kx_d = torch.from_numpy(w["kx"]).to(dev)
        ky_d = torch.from_numpy(w["ky"]).to(dev)
        # simulate the data with the exact forward model on the GPU
        spirec.spirec_set_trajectory_dev(h, kx_d, ky_d)
        f_d = torch.from_numpy(w["f_true"].astype(np.complex64)).to(dev)
        y_d = torch.zeros(L, dtype=torch.complex64, device=dev)
        spirec.spirec_forward_dev(h, f_d, y_d)
        y = y_d.cpu().numpy().astype(np.complex128)
        s = synth.add_noise(y, w["snr"], w["g"]).astype(np.complex64)
        s_d = torch.from_numpy(s).to(dev)
        spirec.spirec_set_reg(h, w["lambda1"], w["alpha1"], w["lambda0"], w["alpha0"], w["phi"])
        x_d = torch.zeros((N, N), dtype=torch.complex64, device=dev)
        J_d = torch.zeros(ITERS + 1, dtype=torch.float64, device=dev)
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

        def step():
            spirec.spirec_set_trajectory_dev(h, kx_d, ky_d)
            spirec.spirec_set_data_dev(h, s_d)
            spirec.spirec_solve_dev(h, None, ITERS, x_d, J_d)

        for _ in range(args.warmup):
            flush.fill_(1.0)
            step()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        spirec.spirec_timing(h, 1)
        l0 = spirec.spirec_launch_count(h)
        proc, cf = clocks_start(torch.cuda.current_device())
        evs = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        clocks = clocks_stop(proc, cf, torch.cuda.current_device())
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        launches = spirec.spirec_launch_count(h) - l0
        stages = spirec.spirec_timing_read(h)
        spirec.spirec_timing(h, 0)
        ms = sum(a.elapsed_time(b) for a, b in evs)
        J = J_d.cpu().numpy()
        x_gpu = x_d.cpu().numpy()

    value, t_s = job_throughput(ms / 1000.0, ITERS * args.steps, dev)

    # ---- end to end through the host-pointer API (pinned buffers)
    kx_h = torch.from_numpy(w["kx"]).pin_memory().numpy()
    ky_h = torch.from_numpy(w["ky"]).pin_memory().numpy()
    s_h = torch.from_numpy(s).pin_memory().numpy()
    xo = torch.zeros((N, N), dtype=torch.complex64).pin_memory().numpy()
    Jo = torch.zeros(ITERS + 1, dtype=torch.float64).pin_memory().numpy()
    lib = spirec.load()
    import ctypes
    e2e_times = []
    for i in range(args.warmup + args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        spirec._check(lib.spirec_set_trajectory(h, ctypes.c_void_p(kx_h.ctypes.data),
                                                ctypes.c_void_p(ky_h.ctypes.data)))
        spirec._check(lib.spirec_set_data(h, ctypes.c_void_p(s_h.ctypes.data)))
        spirec._check(lib.spirec_solve(h, None, ITERS, ctypes.c_void_p(xo.ctypes.data),
                                       ctypes.c_void_p(Jo.ctypes.data)))
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_times.append(t1 - t0)
    e2e_value, _ = job_throughput(sum(e2e_times), ITERS * args.steps, dev)
    spirec.spirec_plan_destroy(h)

    # ---- FP32 plain path on the same workload (the metric's comparison)
    extra = {}
    if prec != spirec.SPIREC_FP32 and not args.no_fp32_compare:
        h2 = spirec.spirec_plan_create(N, L, M, spirec.SPIREC_FP32, stream.cuda_stream)
        with torch.cuda.stream(stream):
            spirec.spirec_set_reg(h2, w["lambda1"], w["alpha1"], w["lambda0"], w["alpha0"], w["phi"])
            x2 = torch.zeros_like(x_d)
            J2 = torch.zeros_like(J_d)
            tt = []
            for i in range(2):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                spirec.spirec_set_trajectory_dev(h2, kx_d, ky_d)
                spirec.spirec_set_data_dev(h2, s_d)
                spirec.spirec_solve_dev(h2, None, ITERS, x2, J2)
                e1.record(stream)
                tt.append((e0, e1))
            torch.cuda.synchronize()
            t2 = tt[1][0].elapsed_time(tt[1][1]) / 1000.0
            xf = x2.cpu().numpy()
            Jf = J2.cpu().numpy()
            # control: the FP32 path again with the trajectory perturbed by
            # 1e-7 (relative, seeded): how far ITERS iterations carry a
            # rounding-sized change of the operators
            pert = 1e-7 * np.random.default_rng(17).standard_normal(L)
            kxp = torch.from_numpy(w["kx"] * (1 + pert)).to(dev)
            kyp = torch.from_numpy(w["ky"] * (1 - pert)).to(dev)
            spirec.spirec_set_trajectory_dev(h2, kxp, kyp)
            spirec.spirec_set_data_dev(h2, s_d)
            spirec.spirec_solve_dev(h2, None, ITERS, x2, J2)
            torch.cuda.synchronize()
            xp = x2.cpu().numpy()
        spirec.spirec_plan_destroy(h2)
        ft = w["f_true"]
        ss = float(np.sum(np.abs(s_d.cpu().numpy().astype(np.complex128)) ** 2))
        extra["fp32_plain_value"] = ITERS / t2
        # the two paths' iterates after ITERS iterations, their criteria (on
        # the scale of ||s||^2, the terms the rewritten criterion cancels), the
        # FP32 path's own spread under a 1e-7 perturbation of k, and each
        # path's distance to the phantom (the reconstruction quality)
        extra["mixed_vs_fp32_rel_l2"] = float(np.linalg.norm(x_gpu - xf) / np.linalg.norm(xf))
        extra["fp32_vs_fp32_k_perturbed_1e-7_rel_l2"] = float(np.linalg.norm(xp - xf) / np.linalg.norm(xf))
        extra["mixed_vs_fp32_J_over_s2"] = float(abs(J[-1] - Jf[-1]) / ss)
        extra["error_to_phantom"] = {"mixed": float(np.linalg.norm(x_gpu - ft) / np.linalg.norm(ft)),
                                     "fp32": float(np.linalg.norm(xf - ft) / np.linalg.norm(ft))}

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return 0

    # ---- many reconstructions: batched dynamic series and a served stream
    if not args.no_batch:
        extra["batch"] = run_batch(spirec, prec)
    if not args.no_paper_experiment:
        extra["paper_experiment"] = run_paper_experiment(spirec, prec)
    if not args.no_direct:
        extra["direct_mode"] = run_direct_mode(spirec, prec, w, s)
    if not args.no_half_quadratic:
        extra["section5_minimisers"] = run_half_quadratic(spirec, prec, w, s)
    if not args.no_graph_path:
        extra["graph_path_2048"] = run_graph_path(spirec, prec, hbm_gbs=(peaks() or {}).get("hbm_gbs"))
    if not args.no_serving:
        extra["serving"] = run_serving(spirec, prec)
        if prec != spirec.SPIREC_FP32 and not args.no_fp32_compare:
            extra["serving_fp32_plain"] = run_serving(spirec, spirec.SPIREC_FP32)

    # ---- roofline of the dominant stage
    pk = peaks()
    dom = max(stages, key=lambda k: stages[k][0])
    dom_ms, dom_n = stages[dom]
    avg_ms = dom_ms / max(dom_n, 1)
    if dom == "gram":
        flops = 8.0 * N * (2 * N - 1) * L
        achieved = flops / (avg_ms / 1000.0) / 1e12
        if prec == spirec.SPIREC_FP32:
            sm_max = (pk or {}).get("sm_max_mhz", 2070.0)
            peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12
            roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None, "kernel": "gram (FP32 CUDA cores)",
                    "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x max SM clock"}
        else:
            peak = (pk or {}).get("bf16_tflops", 1900.0)
            roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": ncu_traffic("k_tc_pair_gemm_G"),
                    "kernel": "gram (tcgen05 FP16x3, k_tc_pair_gemm)",
                    "peak_source": "measured bf16 burst (fp16 dense rate equal)" if pk else "fallback"}
    elif dom == "iterations":
        bytes_ = 160.0 * N * N * ITERS
        achieved = bytes_ / (avg_ms / 1000.0) / 1e9
        peak = (pk or {}).get("hbm_gbs", 6800.0)
        traffic = ncu_traffic("k_cg_loop") if ITERS == 50 and N == 512 else None
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": "CG iteration loop (k_cg_loop)",
                "peak_source": "measured" if pk else "fallback",
                "note": "working set stays in shared memory and L2 across iterations: DRAM traffic "
                        "(ncu, per launch) is 0.5% of the algorithmic bytes"}
    else:
        flops = 8.0 * N * N * L
        achieved = flops / (avg_ms / 1000.0) / 1e12
        peak = (pk or {}).get("bf16_tflops", 1900.0)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": dom}
    roof["stage_ms_per_step"] = {k: v[0] / max(args.steps, 1) for k, v in stages.items()}
    # the contraction beside it: G on the tensor cores, algorithmic flops (the
    # dense count 8 N (2N-1) L of Eq. AnnMatG) and issued MMA flops (pair tiles
    # of 256 rows x 128 paired columns: two accumulators of 256 rows x 256
    # stacked B rows [Br ; Bi], three split products hi*hi + hi*lo + lo*hi
    # each) against the measured bf16 rate
    if prec != spirec.SPIREC_FP32 and stages["gram"][1] > 0:
        g_ms = stages["gram"][0] / stages["gram"][1]
        flops = 8.0 * N * (2 * N - 1) * L
        tiles = ((N + 255) // 256) * ((N + 127) // 128)
        issued = 2.0 * 2 * 3 * 256 * 256 * (32 * ((L + 31) // 32)) * tiles
        peak = (pk or {}).get("bf16_tflops", 1900.0)
        extra["roofline_contraction"] = {
            "bound": "tensor", "kernel": "k_tc_pair_gemm (G) + its split-K sum (k_reduce_pair)", "unit": "TFLOP/s",
            "achieved": flops / (g_ms / 1000.0) / 1e12, "achieved_issued": issued / (g_ms / 1000.0) / 1e12,
            "peak": peak, "frac": flops / (g_ms / 1000.0) / 1e12 / peak,
            "frac_issued": issued / (g_ms / 1000.0) / 1e12 / peak,
            "traffic": ncu_traffic("k_tc_pair_gemm_G") if N == 512 else None,
            "peak_source": "measured bf16 burst (fp16 dense rate equal)" if pk else "fallback"}

    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        O.build()
        cpu = oracle_sample(w, budget_s=args.cpu_budget)
        extra["cpu_baseline_toeplitz"], extra["err_vs_fp64"] = cpu_fp64_leg(spirec, w, dev)

    dtype = {spirec.SPIREC_FP32: "f32", spirec.SPIREC_MIXED_FP16X3: "fp16x3+f32",
             spirec.SPIREC_MIXED_BF16X3: "bf16x3+f32"}[prec]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": w["name"], "precision": args.precision, "iters_per_step": ITERS,
                   "l2": "flushed (256 MB write) before every timed step", "parallelism": f"replicas x{ws}"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(16 * L + 8 * L),
                "d2h_bytes_per_step": int(8 * N * N + 8 * (ITERS + 1) + 4)},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "J_first_last": [float(J[0]), float(J[-1])],
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=os.environ.get("SPIREC_BENCH_PRECISION", "fp16x3"),
                    choices=["fp32", "fp16x3", "bf16x3"])
    ap.add_argument("--no-fp32-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-frame dynamic-series batch")
    ap.add_argument("--no-serving", action="store_true", help="skip the served request stream")
    ap.add_argument("--no-half-quadratic", action="store_true",
                    help="skip the half-quadratic vs PR+ CG comparison at an equal T-apply budget")
    ap.add_argument("--no-graph-path", action="store_true",
                    help="skip the stand-alone-kernel iteration on a 2048^2 image (HBM-bound FFT and stencil kernels)")
    ap.add_argument("--only-graph-path", action="store_true",
                    help="run only that measurement and print its JSON (for profiling its kernels)")
    ap.add_argument("--no-direct", action="store_true",
                    help="skip the per-iteration comparison with the direct (non-rewritten) formulation")
    ap.add_argument("--no-paper-experiment", action="store_true",
                    help="skip the 128x128 two-vessel experiment with the paper's hyperparameters")
    ap.add_argument("--samples", type=int, default=4096,
                    help="samples per interleave (4096 = the metric's 131072-sample spiral)")
    ap.add_argument("--iters", type=int, default=50, help="CG iterations per step (50 = the metric's)")
    args = ap.parse_args()
    apply_size_args(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.only_graph_path:
        import torch
        from paper_0908_3252_gb300 import build, spirec
        build.build()
        spirec.load()
        prec = {"fp32": spirec.SPIREC_FP32, "fp16x3": spirec.SPIREC_MIXED_FP16X3,
                "bf16x3": spirec.SPIREC_MIXED_BF16X3}[args.precision]
        print(json.dumps(run_graph_path(spirec, prec, hbm_gbs=(peaks() or {}).get("hbm_gbs"))))
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
