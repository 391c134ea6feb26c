"""ctypes wrapper around the FP64 CPU oracle (``spirec_oracle.c``).

Test infrastructure only: the tests, the smoke check and the benchmark's CPU
baseline import this module; the product library never does.  The oracle
shares no code with the CUDA path.  Complex arrays cross this wrapper as numpy
``complex128``; images are ``(N, N)`` with axis 0 the row index n (paired with
ky) and axis 1 the column index m (paired with kx), as in Eq. ModDirect.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spirec_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

PHI_HUBER, PHI_HYPERBOLIC, PHI_QUADRATIC = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        i32 = ctypes.c_int32
        i64 = ctypes.c_int64
        pi32 = ctypes.POINTER(ctypes.c_int32)
        _lib.oracle_forward.argtypes = [i32, i64, d, d, d, d]
        _lib.oracle_adjoint.argtypes = [i32, i64, d, d, d, d]
        _lib.oracle_adjoint_at.argtypes = [i32, i64, d, d, d, i64, pi32, pi32, d]
        _lib.oracle_gram.argtypes = [i32, i64, d, d, d]
        _lib.oracle_gram_at.argtypes = [i32, i64, d, d, i64, pi32, pi32, d]
        _lib.oracle_autocorr.argtypes = [i32, d, d]
        _lib.oracle_toeplitz_apply.argtypes = [i32, d, d, d]
        _lib.oracle_phi.argtypes = [i32, ctypes.c_double, ctypes.c_double]
        _lib.oracle_phi.restype = ctypes.c_double
        _lib.oracle_phi_weight.argtypes = [i32, ctypes.c_double, ctypes.c_double]
        _lib.oracle_phi_weight.restype = ctypes.c_double
        _lib.oracle_penalty.argtypes = [i32, d, ctypes.c_void_p]
        _lib.oracle_penalty.restype = ctypes.c_double
        _lib.oracle_penalty_grad.argtypes = [i32, d, ctypes.c_void_p, d]
        _lib.oracle_objective.argtypes = [i32, i64, d, d, d, d, ctypes.c_void_p]
        _lib.oracle_objective.restype = ctypes.c_double
        _lib.oracle_gradient.argtypes = [i32, i64, d, d, d, d, ctypes.c_void_p, d]
        _lib.oracle_solve.argtypes = [i32, i64, d, d, d, ctypes.c_void_p, d, i32, d, d, d]
        _lib.oracle_solve.restype = ctypes.c_int
        _lib.oracle_num_threads.restype = ctypes.c_int
    return _lib


class _Reg(ctypes.Structure):
    _fields_ = [("lambda1", ctypes.c_double), ("alpha1", ctypes.c_double),
                ("lambda0", ctypes.c_double), ("alpha0", ctypes.c_double),
                ("kind", ctypes.c_int32)]


@dataclass
class Reg:
    """R(f) = lambda1 Omega1(f) + lambda0 Omega0(f) with one phi kind (section 3.3)."""
    lambda1: float = 0.0
    alpha1: float = 1.0
    lambda0: float = 0.0
    alpha0: float = 1.0
    kind: int = PHI_HUBER

    def _c(self):
        return _Reg(self.lambda1, self.alpha1, self.lambda0, self.alpha0, self.kind)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _cplx(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a


def _traj(kx, ky):
    kx = np.ascontiguousarray(kx, dtype=np.float64)
    ky = np.ascontiguousarray(ky, dtype=np.float64)
    assert kx.shape == ky.shape and kx.ndim == 1
    return kx, ky


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def forward(kx, ky, f):
    """y = H f (Eq. ModDirect)."""
    kx, ky = _traj(kx, ky)
    f = _cplx(f)
    N = f.shape[0]
    y = np.zeros(kx.shape[0], np.complex128)
    _load().oracle_forward(N, kx.shape[0], _dp(kx), _dp(ky), _dp(f), _dp(y))
    return y


def adjoint(kx, ky, r, N):
    """x = H^H r; with r = s this is D (Eq. AnnMatGD)."""
    kx, ky = _traj(kx, ky)
    r = _cplx(r)
    x = np.zeros((N, N), np.complex128)
    _load().oracle_adjoint(N, kx.shape[0], _dp(kx), _dp(ky), _dp(r), _dp(x))
    return x


def adjoint_at(kx, ky, r, N, n, m):
    """D at sampled pixels (n_i, m_i)."""
    kx, ky = _traj(kx, ky)
    r = _cplx(r)
    n = np.ascontiguousarray(n, np.int32)
    m = np.ascontiguousarray(m, np.int32)
    out = np.zeros(n.shape[0], np.complex128)
    _load().oracle_adjoint_at(N, kx.shape[0], _dp(kx), _dp(ky), _dp(r), n.shape[0], _ip(n), _ip(m), _dp(out))
    return out


def gram(kx, ky, N):
    """Full G (Eq. AnnMatG) as a (2N-1, 2N-1) array indexed [v+N-1, u+N-1]."""
    kx, ky = _traj(kx, ky)
    W = 2 * N - 1
    G = np.zeros((W, W), np.complex128)
    _load().oracle_gram(N, kx.shape[0], _dp(kx), _dp(ky), _dp(G))
    return G


def gram_at(kx, ky, N, u, v):
    """G_{u_i, v_i} at sampled lags."""
    kx, ky = _traj(kx, ky)
    u = np.ascontiguousarray(u, np.int32)
    v = np.ascontiguousarray(v, np.int32)
    out = np.zeros(u.shape[0], np.complex128)
    _load().oracle_gram_at(N, kx.shape[0], _dp(kx), _dp(ky), u.shape[0], _ip(u), _ip(v), _dp(out))
    return out


def autocorr(f):
    """Image correlation C_{u,v} (Appendix A), indexed like G."""
    f = _cplx(f)
    N = f.shape[0]
    C = np.zeros((2 * N - 1, 2 * N - 1), np.complex128)
    _load().oracle_autocorr(N, _dp(f), _dp(C))
    return C


def toeplitz_apply(G, x):
    """T x by direct lag sums with G (Appendix B)."""
    G = _cplx(G)
    x = _cplx(x)
    N = x.shape[0]
    out = np.zeros_like(x)
    _load().oracle_toeplitz_apply(N, _dp(G), _dp(x), _dp(out))
    return out


def phi(kind, alpha, r):
    return float(_load().oracle_phi(kind, alpha, r))


def phi_weight(kind, alpha, r):
    return float(_load().oracle_phi_weight(kind, alpha, r))


def penalty(f, reg: Reg):
    f = _cplx(f)
    c = reg._c()
    return float(_load().oracle_penalty(f.shape[0], _dp(f), ctypes.byref(c)))


def penalty_grad(f, reg: Reg):
    f = _cplx(f)
    g = np.zeros_like(f)
    c = reg._c()
    _load().oracle_penalty_grad(f.shape[0], _dp(f), ctypes.byref(c), _dp(g))
    return g


def objective(kx, ky, s, f, reg: Reg):
    """J(f) = ||s - H f||^2 + R(f) (Eq. CritLS plus the prior)."""
    kx, ky = _traj(kx, ky)
    s = _cplx(s)
    f = _cplx(f)
    c = reg._c()
    return float(_load().oracle_objective(f.shape[0], kx.shape[0], _dp(kx), _dp(ky), _dp(s), _dp(f), ctypes.byref(c)))


def gradient(kx, ky, s, f, reg: Reg):
    """grad J = 2 H^H (H f - s) + grad R (dJ/dRe f + i dJ/dIm f)."""
    kx, ky = _traj(kx, ky)
    s = _cplx(s)
    f = _cplx(f)
    g = np.zeros_like(f)
    c = reg._c()
    _load().oracle_gradient(f.shape[0], kx.shape[0], _dp(kx), _dp(ky), _dp(s), _dp(f), ctypes.byref(c), _dp(g))
    return g


def solve(kx, ky, s, reg: Reg, x0, iters):
    """PR+ CG with three majorize-minimize line-search steps.

    Returns (x, J_hist[iters+1], t_hist[iters])."""
    kx, ky = _traj(kx, ky)
    s = _cplx(s)
    x0 = _cplx(x0)
    N = x0.shape[0]
    x = np.zeros_like(x0)
    J = np.zeros(iters + 1, np.float64)
    t = np.zeros(max(iters, 1), np.float64)
    c = reg._c()
    rc = _load().oracle_solve(N, kx.shape[0], _dp(kx), _dp(ky), _dp(s), ctypes.byref(c), _dp(x0),
                              iters, _dp(x), _dp(J), _dp(t))
    if rc != 0:
        raise MemoryError("oracle_solve failed")
    return x, J, t[:iters]
