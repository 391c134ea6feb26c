"""Shared test helpers: seeded workloads and GPU plumbing (no reconstruction
arithmetic here; expected values always come from the oracle)."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O
from paper_0908_3252_gb300 import synth


def rel(a, b):
    a = np.asarray(a, np.complex128).ravel()
    b = np.asarray(b, np.complex128).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def c64(a):
    """Round to complex64 and back: the exact values the FP32 path receives."""
    return np.asarray(a).astype(np.complex64).astype(np.complex128)


def workload_c1(seed=1):
    """32x32, 10 ellipses (zero phase), Archimedean spiral 4 x 256, 30 dB,
    hyperbolic phi alpha 0.05, lambda1 0.1, 50 iterations."""
    N = 32
    g = synth.rng(seed)
    f_true = synth.phantom(N, "ellipses", g)
    kx, ky = synth.spiral(N, 4, 256, "archimedean")
    s = c64(synth.add_noise(O.forward(kx, ky, f_true), 30.0, g))
    reg = O.Reg(0.1, 0.05, 0.0, 0.05, O.PHI_HYPERBOLIC)
    return dict(N=N, kx=kx, ky=ky, f_true=f_true, s=s, reg=reg, iters=50)


def workload_ragged(N=37, I=3, S=333, seed=7, kind=O.PHI_HUBER):
    """Odd image side and sample count (ragged against every tile size)."""
    g = synth.rng(seed)
    f_true = synth.phantom(N, "ellipses_phase", g)
    kx, ky = synth.spiral(N, I, S, "variable")
    s = c64(synth.add_noise(O.forward(kx, ky, f_true), 25.0, g))
    reg = O.Reg(0.05, 0.05, 0.02, 0.1, kind)
    return dict(N=N, kx=kx, ky=ky, f_true=f_true, s=s, reg=reg, iters=30)


def torch_dev():
    import torch
    return torch.device("cuda:0")


def to_dev(a, dtype="c64"):
    import torch
    if dtype == "c64":
        return torch.from_numpy(np.ascontiguousarray(a, np.complex64)).to(torch_dev())
    return torch.from_numpy(np.ascontiguousarray(a, np.float64)).to(torch_dev())


def from_dev(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def empty_c64(shape):
    import torch
    return torch.zeros(shape, dtype=torch.complex64, device=torch_dev())


_SPREAD = {}


# relative error of the FP32 path's operators against the oracle, measured on
# the 32^2 workload: G 2.8e-7, D 1.8e-7, T 2.7e-7
OPERATOR_NOISE = 3e-7


def fp32_spread(w, x0=None, iters=None, noise=OPERATOR_NOISE, seeds=range(8)):
    """Distances from the FP64 oracle's iterate of the FP32 rounding model
    (oracle/fp32_model.py) after `iters` iterations of the workload: FP32
    storage of every vector, and relative perturbations of `noise` of the
    kernel spectrum, D, every T apply and every gradient (the size of the
    FP32 path's operator errors), one run per seed.  Cached per workload."""
    from oracle import fp32_model as FM
    from oracle import toeplitz_cpu as TC
    N = w["N"]
    iters = w["iters"] if iters is None else iters
    key = (N, w["kx"].shape[0], float(w["kx"][-1]), float(np.abs(w["s"]).sum()), iters, noise,
           None if x0 is None else float(np.abs(x0).sum()))
    if key not in _SPREAD:
        x0c = np.zeros((N, N)) if x0 is None else c64(x0)
        C = TC.kernel_spectrum(O.gram(w["kx"], w["ky"], N), N, 2 * N)
        D = O.adjoint(w["kx"], w["ky"], w["s"], N)
        ss = float(np.sum(np.abs(w["s"]) ** 2))
        xo, _, _ = O.solve(w["kx"], w["ky"], w["s"], w["reg"], x0c, iters)
        _SPREAD[key] = FM.spread(C, D, ss, w["reg"], x0c, iters, xo, noise=noise, seeds=seeds)
    return _SPREAD[key]


def iter_tol(w, prec, x0=None, iters=None):
    """Tolerance of an iterate after many iterations: the path's target (1e-5
    FP32, 1e-3 mixed) or 3 x the largest distance the FP32 rounding model
    shows on the same problem, whichever is larger."""
    target = 1e-5 if prec == 0 else 1e-3
    return max(target, 3.0 * max(fp32_spread(w, x0, iters)))

