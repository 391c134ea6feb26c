"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a library
FFT on the complete Cartesian grid (section 3.1, Eq. InvCart), closed forms,
the identities of Appendix A and B, finite differences, and a dense
normal-equation solve for the quadratic penalty (section 3.3).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0908_3252_gb300 import synth
from tests.helpers import workload_c1, workload_ragged


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def _rand_problem(N, L, seed):
    g = synth.rng(seed)
    kx, ky = synth.uniform_k(L, g)
    f = synth.complex_normal((N, N), g)
    s = synth.complex_normal(L, g)
    return kx, ky, f, s


# ------------------------------------------------------------ Cartesian pins

@pytest.mark.parametrize("N", [8, 12])
def test_cartesian_forward_is_scaled_inverse_fft(N):
    """Complete Cartesian sampling: H is the inverse DFT matrix (section 3.1),
    (Hf)_l = N * ifft2(f)[jy mod N, jx mod N] in numpy's convention."""
    g = synth.rng(11)
    kx, ky = synth.cartesian(N)
    f = synth.complex_normal((N, N), g)
    y = O.forward(kx, ky, f)
    F = N * np.fft.ifft2(f)
    jx = np.rint(kx * N).astype(int) % N
    jy = np.rint(ky * N).astype(int) % N
    assert rel(y, F[jy, jx]) < 1e-12


@pytest.mark.parametrize("N", [8, 10])
def test_cartesian_gram_is_identity(N):
    """H^H H = I on the complete grid (Eq. InvCart): the adjoint inverts the
    forward, and G is a unit impulse at lag (0, 0) with G_00 = L/N^2 = 1."""
    g = synth.rng(12)
    kx, ky = synth.cartesian(N)
    f = synth.complex_normal((N, N), g)
    assert rel(O.adjoint(kx, ky, O.forward(kx, ky, f), N), f) < 1e-12
    G = O.gram(kx, ky, N)
    delta = np.zeros_like(G)
    delta[N - 1, N - 1] = 1.0
    assert np.max(np.abs(G - delta)) < 1e-12


def test_cartesian_unregularized_one_step():
    """lambda = 0, complete grid, noise-free data: J = ||f - f*||^2, so the
    first CG step with the majorize-minimize line search lands on f* exactly."""
    N = 8
    g = synth.rng(13)
    kx, ky = synth.cartesian(N)
    f_true = synth.complex_normal((N, N), g)
    s = O.forward(kx, ky, f_true)
    x, J, t = O.solve(kx, ky, s, O.Reg(0.0, 1.0, 0.0, 1.0, O.PHI_HUBER), np.zeros((N, N)), 1)
    assert rel(x, f_true) < 1e-12
    assert abs(t[0] - 0.5) < 1e-12
    assert J[1] < 1e-20 * max(J[0], 1.0)


# ------------------------------------------------------------ closed forms

def test_single_sample_constant_image_dirichlet():
    """L = 1, f = 1: y = (1/N) prod of two geometric sums
    (1 - e^{i2pi k N}) / (1 - e^{i2pi k})."""
    N = 16
    kx, ky = np.array([0.1234]), np.array([-0.3712])
    y = O.forward(kx, ky, np.ones((N, N)))

    def geo(k):
        z = np.exp(2j * np.pi * k)
        return (1 - z ** N) / (1 - z)

    assert abs(y[0] - geo(kx[0]) * geo(ky[0]) / N) < 1e-12


def test_single_sample_gram_closed_form():
    """L = 1: G_{u,v} = e^{i2pi(kx u + ky v)} / N^2 for every lag."""
    N = 6
    kx, ky = np.array([0.3]), np.array([-0.45])
    G = O.gram(kx, ky, N)
    u = np.arange(-(N - 1), N)
    expect = np.exp(2j * np.pi * (kx[0] * u[None, :] + ky[0] * u[:, None])) / N ** 2
    assert np.max(np.abs(G - expect)) < 1e-14


# ------------------------------------------------------- Appendix A/B identities

def test_adjoint_identity():
    """<H f, r> = <f, H^H r> (Eq. AnnYS: sum_l s_l y_l^* = sum f^* D)."""
    kx, ky, f, r = _rand_problem(10, 300, 21)
    lhs = np.vdot(O.forward(kx, ky, f), r)
    rhs = np.vdot(f, O.adjoint(kx, ky, r, 10))
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_gram_point_symmetry_not_hermitian():
    """G_{-u,-v} = conj G_{u,v}; G_00 = L/N^2.  The transposed relation
    G_{v,u} = conj G_{u,v} (a literal reading of "G^dag = G") fails for a
    general trajectory, which is why only the point symmetry is used."""
    N, L = 7, 200
    kx, ky, _, _ = _rand_problem(N, L, 22)
    G = O.gram(kx, ky, N)
    assert abs(G[N - 1, N - 1] - L / N ** 2) < 1e-12
    assert np.max(np.abs(G[::-1, ::-1] - np.conj(G))) < 1e-13
    assert np.max(np.abs(G.T - np.conj(G))) > 1e-3


def test_toeplitz_lag_sum_equals_normal_operator():
    """T x by lag sums over G equals H^H (H x) (Appendix B)."""
    N, L = 9, 400
    kx, ky, x, _ = _rand_problem(N, L, 23)
    G = O.gram(kx, ky, N)
    assert rel(O.toeplitz_apply(G, x), O.adjoint(kx, ky, O.forward(kx, ky, x), N)) < 1e-12


def test_sum_CG_equals_model_energy():
    """sum_{u,v} C_{u,v} G_{u,v} = sum_l |y_l|^2 (Eq. AnnYY)."""
    N, L = 8, 350
    kx, ky, f, _ = _rand_problem(N, L, 24)
    lhs = np.sum(O.autocorr(f) * O.gram(kx, ky, N))
    rhs = np.sum(np.abs(O.forward(kx, ky, f)) ** 2)
    assert abs(lhs.imag) < 1e-10 * rhs
    assert abs(lhs.real - rhs) < 1e-11 * rhs


def test_rewritten_criterion_equals_direct():
    """Eq. NewCritLS: sum|s|^2 - 2 Re sum f^* D + sum C G equals the direct
    ||s - H f||^2 of Eq. CritLS."""
    N, L = 8, 300
    kx, ky, f, s = _rand_problem(N, L, 25)
    D = O.adjoint(kx, ky, s, N)
    J_new = (np.sum(np.abs(s) ** 2) - 2 * np.real(np.vdot(f, D))
             + np.real(np.sum(O.autocorr(f) * O.gram(kx, ky, N))))
    J_direct = O.objective(kx, ky, s, f, O.Reg())
    assert abs(J_new - J_direct) < 1e-12 * J_direct


def test_gradient_is_2_Tf_minus_2D():
    """dJ_LS/df = 2 f*G - 2 D (section 3.4, Appendix B), with f*G = T f."""
    N, L = 8, 250
    kx, ky, f, s = _rand_problem(N, L, 26)
    G = O.gram(kx, ky, N)
    D = O.adjoint(kx, ky, s, N)
    g = O.gradient(kx, ky, s, f, O.Reg())
    assert rel(g, 2 * O.toeplitz_apply(G, f) - 2 * D) < 1e-12


# ------------------------------------------------------------ penalties

def test_huber_continuity_and_limits():
    """Huber: C^1 at |x| = alpha; quadratic as alpha -> infinity."""
    a = 0.7
    h = 1e-7
    lo, hi = O.phi(0, a, a - h), O.phi(0, a, a + h)
    assert abs(O.phi(0, a, a) - a * a) < 1e-15
    assert abs(hi - lo) < 3 * 2 * a * h
    assert abs((hi - lo) / (2 * h) - 2 * a) < 1e-6
    for r in [0.0, 0.3, 5.0, 123.0]:
        assert O.phi(0, 1e9, r) == O.phi(2, 0.0, r) == r * r
    # weight b(r) = phi'(r)/r: 2 inside, 2 alpha / r outside
    assert O.phi_weight(0, a, 0.5 * a) == 2.0
    assert abs(O.phi_weight(0, a, 4 * a) - 0.5) < 1e-15


def test_hyperbolic_asymptotes():
    """2a(sqrt(a^2+r^2)-a): ~ r^2 near 0, ~ 2a r - 2a^2 for r >> a, b(0) = 2."""
    a = 0.05
    assert abs(O.phi(1, a, 1e-4) / 1e-8 - 1.0) < 1e-5
    r = 1e4
    assert abs(O.phi(1, a, r) - (2 * a * r - 2 * a * a)) < 1e-6
    assert O.phi_weight(1, a, 0.0) == 2.0


@pytest.mark.parametrize("kind,alpha", [(0, 0.37), (1, 0.05), (2, 1.0)])
def test_gradient_matches_finite_differences(kind, alpha):
    """Full grad J (data + both penalty terms) against central differences
    along the real and imaginary parts of random directions."""
    N, L = 6, 120
    kx, ky, f, s = _rand_problem(N, L, 27 + kind)
    reg = O.Reg(0.3, alpha, 0.2, 1.3 * alpha, kind)
    g = O.gradient(kx, ky, s, f, reg)
    rg = synth.rng(99)
    for _ in range(4):
        v = synth.complex_normal((N, N), rg)
        h = 1e-6
        fd = (O.objective(kx, ky, s, f + h * v, reg) - O.objective(kx, ky, s, f - h * v, reg)) / (2 * h)
        an = np.real(np.vdot(v, g))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


def test_penalty_gradient_boundary_and_sign():
    """Free boundary: a single nonzero pixel in a corner has 2 edges, one in
    the interior 4; quadratic phi gives the discrete Laplacian stencil."""
    N = 5
    f = np.zeros((N, N), np.complex128)
    f[0, 0] = 1.0
    f[2, 2] = 1.0j
    g = O.penalty_grad(f, O.Reg(1.0, 1.0, 0.0, 1.0, O.PHI_QUADRATIC))
    assert g[0, 0] == 2 * 2.0 and g[0, 1] == -2.0 and g[1, 0] == -2.0
    assert g[2, 2] == 4 * 2.0j and g[1, 2] == -2.0j and g[2, 3] == -2.0j
    assert O.penalty(f, O.Reg(1.0, 1.0, 0.0, 1.0, O.PHI_QUADRATIC)) == 2 + 4


# ------------------------------------------------------------ minimiser

def test_quadratic_phi_matches_dense_normal_equations():
    """Quadratic phi (Hunt, section 3.3) on an 8x8 image: the minimiser of
    ||s-Hf||^2 + l1 ||Delta f||^2 + l0 ||f||^2 solves
    (H^H H + l1 Delta^H Delta + l0 I) f = H^H s; CG reaches the LU solution."""
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
    x, J, _ = O.solve(kx, ky, s, O.Reg(l1, 1.0, l0, 1.0, O.PHI_QUADRATIC), np.zeros((N, N)), 400)
    assert rel(x, f_star) < 1e-9
    assert np.all(np.diff(J) <= 1e-12 * J[0])


@pytest.mark.parametrize("kind", [0, 1])
def test_objective_monotone(kind):
    """J(f_k) never increases (majorize-minimize steps, section 3.3)."""
    N = 12
    g = synth.rng(40 + kind)
    kx, ky = synth.spiral(N, 3, 60)
    f_true = synth.phantom(N, "ellipses_phase", g)
    s = synth.add_noise(O.forward(kx, ky, f_true), 30.0, g)
    reg = O.Reg(0.1, 0.05, 0.01, 0.1, kind)
    x, J, t = O.solve(kx, ky, s, reg, np.zeros((N, N)), 25)
    assert np.all(np.diff(J) <= 1e-12 * J[0])
    assert J[-1] < 0.5 * J[0]
    assert abs(J[-1] - O.objective(kx, ky, s, x, reg)) < 1e-10 * J[-1]


@pytest.mark.parametrize("wname", ["c1", "ragged"])
def test_rewritten_criterion_solve_equals_direct_solve(wname):
    """Section 3.4 and Appendix B in FP64: the minimiser run on the rewritten
    criterion, with H^H H applied as the zero-padded FFT convolution with the
    kernel built from G (oracle/toeplitz_cpu.py), reaches the same 50
    iterates and J history as the direct form (oracle.solve, which runs the
    exact NUDFTs every iteration)."""
    from oracle import toeplitz_cpu as TC
    w = workload_c1() if wname == "c1" else workload_ragged()
    N = w["N"]
    kx, ky, s, reg = w["kx"], w["ky"], w["s"], w["reg"]
    M = 1 << int(np.ceil(np.log2(2 * N - 1)))
    Ch = TC.kernel_spectrum(O.gram(kx, ky, N), N, M)
    D = O.adjoint(kx, ky, s, N)
    x, J = TC.solve(Ch, D, float(np.sum(np.abs(s) ** 2)), reg, np.zeros((N, N)), 50)
    xo, Jo, _ = O.solve(kx, ky, s, reg, np.zeros((N, N)), 50)
    assert rel(J, Jo) < 1e-12
    assert rel(x, xo) < 1e-9
    xr = synth.complex_normal((N, N), synth.rng(9))
    assert rel(TC.toeplitz_apply(Ch, xr), O.adjoint(kx, ky, O.forward(kx, ky, xr), N)) < 1e-13
