"""Pins of the half-quadratic oracle (oracle/halfquad.py) against facts that
do not come from it: a dense normal-equation solve, the C oracle's criterion
and gradient (themselves pinned by finite differences), the majorant
property, monotone descent, and the minimiser the PR+ CG oracle reaches."""
import numpy as np
import pytest

from oracle import halfquad as HQ
from oracle import oracle as O
from paper_0908_3252_gb300 import synth


def rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _problem(N, I, S, seed):
    g = synth.rng(seed)
    kx, ky = synth.spiral(N, I, S)
    f = synth.phantom(N, "ellipses_phase", g) if N >= 16 else synth.complex_normal((N, N), g)
    s = O.forward(kx, ky, f) + 0.05 * synth.complex_normal(kx.shape[0], g)
    return kx, ky, s, g


def test_quadratic_phi_one_step_solves_the_dense_normal_equations():
    """Quadratic phi has constant weights W = lambda (phi'(r) / 2r = 1), so one
    outer step with 2 N^2 inner steps (the real dimension) solves
    (H^H H + l1 Delta^H Delta + l0 I) f = H^H s built densely here."""
    N, L = 8, 40
    g = synth.rng(31)
    kx, ky = synth.spiral(N, 2, 20)
    s = synth.complex_normal(L, g)
    l1, l0 = 0.3, 0.05
    P = N * N
    H = np.zeros((L, P), np.complex128)
    for j in range(P):
        e = np.zeros(P, np.complex128)
        e[j] = 1.0
        H[:, j] = O.forward(kx, ky, e.reshape(N, N))
    rows = []
    for n in range(N):
        for m in range(N):
            p = n * N + m
            if n + 1 < N:
                r = np.zeros(P)
                r[p + N], r[p] = 1, -1
                rows.append(r)
            if m + 1 < N:
                r = np.zeros(P)
                r[p + 1], r[p] = 1, -1
                rows.append(r)
    Dl = np.array(rows)
    A = H.conj().T @ H + l1 * Dl.T @ Dl + l0 * np.eye(P)
    f_star = np.linalg.solve(A, H.conj().T @ s).reshape(N, N)
    x, J = HQ.solve(kx, ky, s, O.Reg(l1, 1.0, l0, 1.0, O.PHI_QUADRATIC), np.zeros((N, N)), 1, 2 * P)
    assert rel(x, f_star) < 1e-9
    assert J[1] <= J[0]


@pytest.mark.parametrize("kind", [O.PHI_HUBER, O.PHI_HYPERBOLIC])
def test_weights_make_a_tangent_majorant(kind):
    """At f^k the surrogate equals J and its gradient 2 (H^H (H f - s) +
    sum W delta^H delta f) equals the C oracle's gradient; elsewhere it lies
    above J.  A dropped term, a wrong factor or sign in the weights or the
    stencil breaks one of these."""
    N = 10
    kx, ky, s, g = _problem(N, 2, 60, 51 + kind)
    reg = O.Reg(0.4, 0.3, 0.2, 0.5, kind)
    fk = synth.complex_normal((N, N), g)
    Jk = O.objective(kx, ky, s, fk, reg)
    assert abs(HQ.surrogate(kx, ky, s, fk, fk, reg) - Jk) < 1e-12 * Jk
    W = HQ.weights(fk, reg)
    grad_q = 2.0 * (O.adjoint(kx, ky, O.forward(kx, ky, fk) - s, N) + HQ.penalty_normal(fk, W))
    assert rel(grad_q, O.gradient(kx, ky, s, fk, reg)) < 1e-11
    for scale in [1e-3, 0.1, 1.0, 10.0]:
        f = fk + scale * synth.complex_normal((N, N), g)
        assert HQ.surrogate(kx, ky, s, f, fk, reg) >= O.objective(kx, ky, s, f, reg) - 1e-12 * Jk


@pytest.mark.parametrize("kind", [O.PHI_HUBER, O.PHI_HYPERBOLIC])
def test_criterion_never_increases(kind):
    N = 16
    kx, ky, s, g = _problem(N, 3, 80, 61 + kind)
    reg = O.Reg(0.3, 0.1, 0.05, 0.2, kind)
    _, J = HQ.solve(kx, ky, s, reg, np.zeros((N, N)), 15, 3)
    assert np.all(np.diff(J) <= 1e-12 * J[0])
    assert J[-1] < 0.5 * J[0]


def test_reaches_the_minimiser_of_the_conjugate_gradient_oracle():
    """Hyperbolic phi on the pixels makes J strictly convex: the half-
    quadratic iterates and the PR+ CG oracle's converge to one minimiser,
    where the C oracle's gradient vanishes."""
    N = 10
    kx, ky, s, g = _problem(N, 4, 60, 71)
    reg = O.Reg(0.3, 0.2, 0.1, 0.3, O.PHI_HYPERBOLIC)
    x0 = np.zeros((N, N))
    xh, Jh = HQ.solve(kx, ky, s, reg, x0, 80, 12)
    xc, Jc, _ = O.solve(kx, ky, s, reg, x0, 600)
    g0 = np.linalg.norm(O.gradient(kx, ky, s, x0, reg))
    assert np.linalg.norm(O.gradient(kx, ky, s, xh, reg)) < 1e-8 * g0
    assert rel(xh, xc) < 1e-7
    assert abs(Jh[-1] - Jc[-1]) < 1e-12 * Jc[0]
