"""Pins of the truncated-Newton oracle (oracle/newton.py) against facts that
do not come from it: central differences of the C oracle's phi' and
gradient, a dense normal-equation solve, monotone descent, and the minimiser
the PR+ CG oracle reaches."""
import numpy as np
import pytest

from oracle import newton as NT
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


@pytest.mark.parametrize("kind", [O.PHI_HUBER, O.PHI_HYPERBOLIC, O.PHI_QUADRATIC])
def test_phi_second_is_the_derivative_of_the_c_oracles_phi_prime(kind):
    """phi'(r) = r b(r) from the C oracle; its central difference is phi''
    (away from Huber's kink at r = alpha), and e(r) (phi'' - b) / r^2."""
    alpha, h = 0.3, 1e-6
    for r in [0.01, 0.1, 0.25, 0.4, 1.0, 3.0]:
        dp = ((r + h) * O.phi_weight(kind, alpha, r + h) - (r - h) * O.phi_weight(kind, alpha, r - h)) / (2 * h)
        assert abs(NT.phi_second(kind, alpha, r) - dp) < 1e-6 * max(1.0, abs(dp))
        e = (dp - O.phi_weight(kind, alpha, r)) / (r * r)
        assert abs(NT.curvature_e(kind, alpha, r) - e) < 1e-4 * max(1.0, abs(e))
    assert NT.curvature_e(kind, alpha, 0.0) == pytest.approx(
        {O.PHI_HUBER: 0.0, O.PHI_HYPERBOLIC: -2.0 / alpha ** 2, O.PHI_QUADRATIC: 0.0}[kind])


@pytest.mark.parametrize("kind", [O.PHI_HUBER, O.PHI_HYPERBOLIC])
def test_hessian_apply_is_the_derivative_of_the_gradient(kind):
    """(grad J(f + h v) - grad J(f - h v)) / 2h against Hess J(f) v, with the
    C oracle's gradient; a dropped term, factor or transposed stencil fails."""
    N = 8
    kx, ky, s, g = _problem(N, 2, 40, 81 + kind)
    reg = O.Reg(0.4, 0.3, 0.2, 0.5, kind)
    f = synth.complex_normal((N, N), g)
    v = synth.complex_normal((N, N), g)
    h = 1e-6
    fd = (O.gradient(kx, ky, s, f + h * v, reg) - O.gradient(kx, ky, s, f - h * v, reg)) / (2 * h)
    assert rel(NT.hessian_apply(kx, ky, f, v, reg), fd) < 1e-6
    # symmetric in the real inner product
    u = synth.complex_normal((N, N), g)
    a = np.sum((NT.hessian_apply(kx, ky, f, v, reg).conj() * u).real)
    b = np.sum((NT.hessian_apply(kx, ky, f, u, reg).conj() * v).real)
    assert abs(a - b) < 1e-10 * max(abs(a), 1.0)


def test_quadratic_phi_one_step_solves_the_dense_normal_equations():
    """Quadratic phi: J is quadratic, so one Newton step with 2 N^2 inner
    steps (the real dimension) and the exact majorize-minimize step (t = 1)
    reach the solution of (H^H H + l1 Delta^H Delta + l0 I) f = H^H s."""
    N, L = 8, 40
    g = synth.rng(32)
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
    x, J = NT.solve(kx, ky, s, O.Reg(l1, 1.0, l0, 1.0, O.PHI_QUADRATIC), np.zeros((N, N)), 1, 2 * P)
    assert rel(x, f_star) < 1e-9
    assert J[1] <= J[0]


@pytest.mark.parametrize("kind", [O.PHI_HUBER, O.PHI_HYPERBOLIC])
def test_criterion_never_increases(kind):
    N = 16
    kx, ky, s, g = _problem(N, 3, 80, 91 + kind)
    reg = O.Reg(0.3, 0.1, 0.05, 0.2, kind)
    _, J = NT.solve(kx, ky, s, reg, np.zeros((N, N)), 10, 4)
    assert np.all(np.diff(J) <= 1e-12 * J[0])
    assert J[-1] < 0.5 * J[0]


def test_reaches_the_minimiser_of_the_conjugate_gradient_oracle():
    """Hyperbolic phi on the pixels makes J strictly convex: the truncated
    Newton iterates and the PR+ CG oracle's converge to one minimiser, where
    the C oracle's gradient vanishes; Newton needs far fewer outer steps."""
    N = 10
    kx, ky, s, g = _problem(N, 4, 60, 72)
    reg = O.Reg(0.3, 0.2, 0.1, 0.3, O.PHI_HYPERBOLIC)
    x0 = np.zeros((N, N))
    xn, Jn = NT.solve(kx, ky, s, reg, x0, 15, 40)
    xc, Jc, _ = O.solve(kx, ky, s, reg, x0, 600)
    g0 = np.linalg.norm(O.gradient(kx, ky, s, x0, reg))
    assert np.linalg.norm(O.gradient(kx, ky, s, xn, reg)) < 1e-8 * g0
    assert rel(xn, xc) < 1e-7
    assert abs(Jn[-1] - Jc[-1]) < 1e-12 * Jc[0]
