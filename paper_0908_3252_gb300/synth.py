"""Seeded synthetic inputs: phantoms, spiral trajectories and noise.

This module only draws inputs.  It holds none of the reconstruction's
arithmetic (no Fourier operator, no penalty, no minimiser), so both the CPU
oracle and the CUDA path can take their inputs from it.  The paper's own
phantom (section 4.1) and acquisitions (section 4.2) are not available, so the
recipes below stand in for them with the same kind of structure:

* ellipse phantoms (additive ellipses, optional smooth complex phase),
* bars of 2-4 px width at random orientations plus fine texture,
* two vessels with parabolic and blunt flow phase on a variable background,
* Archimedean, variable-density and golden-angle interleaved spirals with
  |k| <= 0.5 cycles/pixel (section 2 normalises k to [-0.5, 0.5]),
* circular complex Gaussian noise scaled to an SNR in dB.

Images are complex ``(N, N)`` arrays: axis 0 is the row index n (ky), axis 1
the column index m (kx).  Pixel centres are uncentred integers 0..N-1.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def _grid(N):
    n, m = np.meshgrid(np.arange(N, dtype=np.float64), np.arange(N, dtype=np.float64), indexing="ij")
    return n, m


def ellipses(N: int, count: int, g: np.random.Generator) -> np.ndarray:
    """Sum of `count` filled ellipses: centres U[-0.4,0.4]*N about the image
    centre, semi-axes U[0.05,0.3]*N, angle U[0,pi), intensity U[0,1]."""
    n, m = _grid(N)
    y = n - (N - 1) / 2.0
    x = m - (N - 1) / 2.0
    img = np.zeros((N, N), np.float64)
    for _ in range(count):
        cx, cy = g.uniform(-0.4, 0.4, 2) * N
        a, b = g.uniform(0.05, 0.3, 2) * N
        th = g.uniform(0.0, np.pi)
        amp = g.uniform(0.0, 1.0)
        xr = (x - cx) * np.cos(th) + (y - cy) * np.sin(th)
        yr = -(x - cx) * np.sin(th) + (y - cy) * np.cos(th)
        img += amp * (((xr / a) ** 2 + (yr / b) ** 2) <= 1.0)
    return img


def smooth_phase(N: int, g: np.random.Generator) -> np.ndarray:
    """exp(i pi p(x, y)) with p a random quadratic polynomial, coefficients
    U[-0.5, 0.5], on coordinates normalised to [-1, 1]."""
    n, m = _grid(N)
    y = 2.0 * n / max(N - 1, 1) - 1.0
    x = 2.0 * m / max(N - 1, 1) - 1.0
    c = g.uniform(-0.5, 0.5, 6)
    p = c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * x * y + c[5] * y * y
    return np.exp(1j * np.pi * p)


def bars(N: int, count: int, g: np.random.Generator) -> np.ndarray:
    """`count` bars: length U[20,120] px, width U{2,3,4} px, angle U[0,pi),
    intensity U[0.2,1], centres uniform over the image."""
    n, m = _grid(N)
    img = np.zeros((N, N), np.float64)
    for _ in range(count):
        length = g.uniform(20.0, 120.0)
        width = float(g.integers(2, 5))
        th = g.uniform(0.0, np.pi)
        amp = g.uniform(0.2, 1.0)
        cx, cy = g.uniform(0.0, N - 1, 2)
        along = (m - cx) * np.cos(th) + (n - cy) * np.sin(th)
        across = -(m - cx) * np.sin(th) + (n - cy) * np.cos(th)
        img += amp * ((np.abs(along) <= length / 2) & (np.abs(across) <= width / 2))
    return img


def phantom(N: int, kind: str, g: np.random.Generator) -> np.ndarray:
    """Complex phantoms of the three single-image workloads.

    'ellipses'       10 ellipses, zero phase.
    'ellipses_phase' 10 ellipses times a smooth complex phase.
    'edges_texture'  10 ellipses times a smooth phase, plus 40 bars and
                     uniform texture U[-0.05, 0.05]."""
    if kind == "ellipses":
        return ellipses(N, 10, g).astype(np.complex128)
    if kind == "ellipses_phase":
        return ellipses(N, 10, g) * smooth_phase(N, g)
    if kind == "edges_texture":
        base = ellipses(N, 10, g) * smooth_phase(N, g)
        return base + bars(N, 40, g) + g.uniform(-0.05, 0.05, (N, N))
    raise ValueError(kind)


def vessels(N: int = 128) -> tuple[np.ndarray, dict]:
    """Two vessels on a variable background, the kind of object of the
    paper's simulated model (section 4.1; its exact phantom is not
    available): magnitude with homogeneous regions and sharp edges on an
    intensity scale of about 255, zero phase outside the vessels, a parabolic
    flow profile in one vessel and a blunt one in the other.

    Background 60 + 40 x (x = m / N), a tissue square [0.3, 0.7]^2 at 120,
    vessel 1 (parabolic) centred at (row 0.5, col 0.45), radius 0.12 N,
    vessel 2 (blunt) at (row 0.25, col 0.75), radius 0.10 N, both at 220;
    phase (pi/2)(1 - (r/R)^2) and (pi/2)(1 - (r/R)^8).  Returns the image and
    two masks: 'roi1' the central square [0.35, 0.65]^2, 'roi2' the inner
    disk (r < 0.7 R) of the blunt vessel, where the magnitude is constant."""
    n, m = _grid(N)
    y, x = n / N, m / N
    mag = 60.0 + 40.0 * x
    tissue = (np.abs(x - 0.5) <= 0.2) & (np.abs(y - 0.5) <= 0.2)
    mag = np.where(tissue, 120.0, mag)
    phase = np.zeros((N, N))
    roi2 = np.zeros((N, N), bool)
    for (cy, cx, R, power) in ((0.5, 0.45, 0.12, 2), (0.25, 0.75, 0.10, 8)):
        r = np.hypot(y - cy, x - cx) / R
        inside = r <= 1.0
        mag = np.where(inside, 220.0, mag)
        phase = np.where(inside, 0.5 * np.pi * (1.0 - r ** power), phase)
        if power == 8:
            roi2 = r < 0.7
    roi1 = (np.abs(x - 0.5) <= 0.15) & (np.abs(y - 0.5) <= 0.15)
    return mag * np.exp(1j * phase), {"roi1": roi1, "roi2": roi2}


def spiral(N: int, interleaves: int, samples: int, kind: str = "archimedean",
           rotation: str = "uniform") -> tuple[np.ndarray, np.ndarray]:
    """Interleaved spiral: k(t) = r(t) exp(i (2 pi W t + phi_j)), t = s/(S-1).

    r(t) = 0.5 t (Archimedean) or 0.5 t^1.5 (variable density); W = N/(2I)
    turns, which gives radial spacing 1/N between arms; phi_j = 2 pi j / I
    ('uniform') or j pi (3 - sqrt 5) ('golden').  Returns (kx, ky) of length
    I*S, interleave-major, all with |k| <= 0.5."""
    t = np.arange(samples, dtype=np.float64) / max(samples - 1, 1)
    r = 0.5 * t if kind == "archimedean" else 0.5 * t ** 1.5
    turns = N / (2.0 * interleaves)
    kx, ky = [], []
    for j in range(interleaves):
        rot = 2.0 * np.pi * j / interleaves if rotation == "uniform" else j * np.pi * (3.0 - np.sqrt(5.0))
        ang = 2.0 * np.pi * turns * t + rot
        kx.append(r * np.cos(ang))
        ky.append(r * np.sin(ang))
    kx = np.clip(np.concatenate(kx), -0.5, 0.5)
    ky = np.clip(np.concatenate(ky), -0.5, 0.5)
    return kx, ky


def cartesian(N: int) -> tuple[np.ndarray, np.ndarray]:
    """The complete Cartesian grid k = (jx/N, jy/N), j = -N/2..N/2-1 (N even),
    ky-major order (l = (jy + N/2) * N + (jx + N/2))."""
    j = (np.arange(N) - N // 2) / N
    ky, kx = np.meshgrid(j, j, indexing="ij")
    return kx.ravel().astype(np.float64), ky.ravel().astype(np.float64)


def uniform_k(L: int, g: np.random.Generator) -> tuple[np.ndarray, np.ndarray]:
    """L points uniform in [-0.5, 0.5]^2."""
    return g.uniform(-0.5, 0.5, L), g.uniform(-0.5, 0.5, L)


def complex_normal(shape, g: np.random.Generator) -> np.ndarray:
    """Circular complex Gaussian, E|w|^2 = 1 (real and imaginary parts each of
    variance 1/2)."""
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)) / np.sqrt(2.0)


def noise_sigma(clean: np.ndarray, snr_db: float) -> float:
    """sigma with sigma^2 = mean |clean|^2 / 10^(SNR/10)."""
    return float(np.sqrt(np.mean(np.abs(clean) ** 2) / 10.0 ** (snr_db / 10.0)))


def add_noise(clean: np.ndarray, snr_db: float, g: np.random.Generator) -> np.ndarray:
    return clean + noise_sigma(clean, snr_db) * complex_normal(clean.shape, g)
