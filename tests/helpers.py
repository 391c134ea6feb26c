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
