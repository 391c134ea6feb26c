"""FP32 rounding model of the PR+ CG minimiser: how far a single-precision
implementation of the same method lands from the FP64 oracle.

TEST INFRASTRUCTURE ONLY.  Nothing in the product library imports or calls
this module; only the tests and the benchmark's CPU leg do.  It shares no code
with the CUDA path.

The minimiser is that of oracle.solve and toeplitz_cpu.solve (section 3.3:
Polak-Ribiere with a descent restart, three majorize-minimize line-search
steps on h(t) = J(f + t d)) on the rewritten criterion of section 3.4:
    grad J(f) = 2 (T f - D) + grad R(f),
    J(f)      = ||s||^2 - 2 Re<f, D> + Re<f, T f> + R(f).
It carries res = T f - D from one iteration to the next (res += t T d), as a
single-precision implementation does to keep the rounding of the data term's
gradient relative to res rather than to D.  Every vector such an
implementation stores is rounded to FP32 where it is formed: D, the kernel
spectrum, the iterate f, the direction d, the gradient g, res and T d.  Dot
products, line-search sums and step sizes stay FP64.  Optionally each T apply,
each gradient, D and the kernel spectrum also carry a seeded relative
perturbation of size `noise` per element, standing in for the rounding inside
FP32 FFTs, stencils and contractions.

With fp32=False and noise=0 nothing is rounded and the model is the FP64
minimiser (pinned to oracle.solve in tests/test_oracle_fp32_model_pins.py).
`deviations` (and `spread`) run several perturbation seeds and return each
run's relative L2 distance to a reference iterate (and the largest difference
of the J histories): the spread an FP32 implementation of the method can show
on that problem after that many iterations.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as O
from oracle import toeplitz_cpu as TC


def fl32(a) -> np.ndarray:
    """Round to the nearest single-precision complex value (kept as complex128)."""
    return np.asarray(a).astype(np.complex64).astype(np.complex128)


def _perturb(a, noise, rng):
    if noise == 0.0 or rng is None:
        return a
    e = rng.standard_normal(a.shape) + 1j * rng.standard_normal(a.shape)
    return a * (1.0 + noise * e)


def solve(C_hat, D, ss, reg: O.Reg, x0, iters, fp32=True, noise=0.0, seed=None):
    """The minimiser with FP32 storage (fp32) and per-evaluation perturbations
    (noise, seeded).  C_hat from toeplitz_cpu.kernel_spectrum, D = H^H s,
    ss = ||s||^2.  Returns (x, J_hist)."""
    rng = np.random.default_rng(seed) if noise else None
    R = fl32 if fp32 else (lambda a: np.asarray(a, np.complex128))
    if fp32 or noise:
        C_hat = np.real(_perturb(np.real(C_hat).astype(np.complex128), noise, rng))
        if fp32:
            C_hat = C_hat.astype(np.float32).astype(np.float64)
    D = R(_perturb(np.asarray(D, np.complex128), noise, rng))
    f = R(np.array(x0, np.complex128))
    res = R(_perturb(TC.toeplitz_apply(C_hat, f), noise, rng) - D)

    def grad_and_J(f, res):
        g = R(_perturb(2.0 * res + O.penalty_grad(f, reg), noise, rng))
        J = ss - TC._redot(f, D) + TC._redot(f, res) + O.penalty(f, reg)
        return g, J

    g, J = grad_and_J(f, res)
    Js = [J]
    d = -g
    for _ in range(iters):
        Td = R(_perturb(TC.toeplitz_apply(C_hat, d), noise, rng))
        q2 = TC._redot(d, Td)
        q1 = 2.0 * TC._redot(d, res)
        t = 0.0
        for _ in range(3):
            num, den = TC._line_terms(f, d, t, reg)
            num += q1 + 2.0 * q2 * t
            den += 2.0 * q2
            if den > 0.0:
                t -= num / den
        f = R(f + t * d)
        res = R(res + t * Td)
        gn, J = grad_and_J(f, res)
        Js.append(J)
        gg_old = TC._redot(g, g)
        beta = max(0.0, TC._redot(gn, gn - g) / gg_old) if gg_old > 0.0 else 0.0
        d = R(-gn + beta * d)
        if TC._redot(gn, d) >= 0.0:
            d = -gn
        g = gn
    return f, np.array(Js)


def deviations(C_hat, D, ss, reg: O.Reg, x0, iters, x_ref, J_ref=None, noise=1e-7, seeds=range(8)):
    """The FP32 model after `iters` iterations against a reference run: per
    run (the unperturbed one first, then one per seed) the relative L2
    distance of the iterate to x_ref and, with J_ref, the largest absolute
    difference of the J histories.  Returns (x_distances, J_differences)."""
    nref = max(np.linalg.norm(x_ref), 1e-300)
    xd, jd = [], []
    for sd in [None] + list(seeds):
        x, J = solve(C_hat, D, ss, reg, x0, iters, fp32=True, noise=0.0 if sd is None else noise, seed=sd)
        xd.append(float(np.linalg.norm(x - x_ref) / nref))
        if J_ref is not None:
            jd.append(float(np.max(np.abs(J - np.asarray(J_ref)))))
    return xd, jd


def spread(C_hat, D, ss, reg: O.Reg, x0, iters, x_ref, noise=1e-7, seeds=range(8)):
    """Relative L2 distance to x_ref of the FP32 model after `iters`
    iterations: the unperturbed run first, then one run per seed."""
    return deviations(C_hat, D, ss, reg, x0, iters, x_ref, None, noise, seeds)[0]
