"""Python binding of libspirec.so (argument marshalling only).

Every function named ``spirec_*`` here calls the C entry point of the same
name in ``include/spirec.h`` through ctypes; no step of the reconstruction
runs in Python.  Host-pointer entry points take numpy arrays (``complex64`` for
complex data, ``float64`` for trajectories); ``*_dev`` entry points take CUDA
tensors (torch is used only to own device memory and streams).

The library must have been built (``paper_0908_3252_gb300.build.build()``);
importing this module without it raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspirec.so")

SPIREC_OK = 0
SPIREC_EINVAL = -1
SPIREC_ENOMEM = -2
SPIREC_ECUDA = -3
SPIREC_ESTATE = -4
SPIREC_EBUSY = -5
SPIREC_ETIMEOUT = -6
SPIREC_ENUMERIC = -7
SPIREC_EUNSUPPORTED = -8

SPIREC_FP32 = 0
SPIREC_MIXED_FP16X3 = 1
SPIREC_MIXED_BF16X3 = 2

SPIREC_PHI_HUBER = 0
SPIREC_PHI_HYPERBOLIC = 1
SPIREC_PHI_QUADRATIC = 2
SPIREC_MODE_TOEPLITZ = 0
SPIREC_MODE_DIRECT = 1

SPIREC_MIN_PRCG = 0
SPIREC_MIN_HALF_QUADRATIC = 1
SPIREC_MIN_NEWTON = 2

SPIREC_KNOB_GRAM_SPLIT = 0
SPIREC_KNOB_ADJOINT_SPLIT = 1
SPIREC_KNOB_LOOP_ROWS = 2
SPIREC_KNOB_GRAM_TILE = 3
SPIREC_KNOB_ADJOINT_TILE = 4
SPIREC_NUM_KNOBS = 5
SPIREC_TUNE_LATENCY = 0
SPIREC_TUNE_THROUGHPUT = 1

SPIREC_NUM_STAGES = 4
STAGES = ("gram", "spectrum", "adjoint_d", "iterations")

# name -> (restype, argtypes) for every symbol declared in include/spirec.h
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double
SIGNATURES = {
    "spirec_plan_create": (ctypes.c_int, [ctypes.POINTER(_P), _I32, _I64, _I32, _I32, _P, _P, _P]),
    "spirec_plan_destroy": (ctypes.c_int, [_P]),
    "spirec_set_trajectory": (ctypes.c_int, [_P, _P, _P]),
    "spirec_set_trajectory_dev": (ctypes.c_int, [_P, _P, _P]),
    "spirec_set_data": (ctypes.c_int, [_P, _P]),
    "spirec_set_data_dev": (ctypes.c_int, [_P, _P]),
    "spirec_set_reg": (ctypes.c_int, [_P, _D, _D, _D, _D, _I32]),
    "spirec_set_mode": (ctypes.c_int, [_P, _I32]),
    "spirec_set_minimiser": (ctypes.c_int, [_P, _I32, _I32]),
    "spirec_kcache_create": (ctypes.c_int, [ctypes.POINTER(_P), _I32, _I32, _I32, _I32, _P, _P, _P, _P]),
    "spirec_kcache_destroy": (ctypes.c_int, [_P]),
    "spirec_set_trajectory_cached": (ctypes.c_int, [_P, _P, _P, _I32]),
    "spirec_solve": (ctypes.c_int, [_P, _P, _I32, _P, _P]),
    "spirec_solve_dev": (ctypes.c_int, [_P, _P, _I32, _P, _P]),
    "spirec_forward_dev": (ctypes.c_int, [_P, _P, _P]),
    "spirec_adjoint_dev": (ctypes.c_int, [_P, _P, _P]),
    "spirec_gram_dev": (ctypes.c_int, [_P, _P]),
    "spirec_kernel_spectrum_dev": (ctypes.c_int, [_P, _P]),
    "spirec_data_adjoint_dev": (ctypes.c_int, [_P, _P]),
    "spirec_toeplitz_dev": (ctypes.c_int, [_P, _P, _P]),
    "spirec_objective_grad_dev": (ctypes.c_int, [_P, _P, _P, _P]),
    "spirec_forward": (ctypes.c_int, [_P, _P, _P]),
    "spirec_adjoint": (ctypes.c_int, [_P, _P, _P]),
    "spirec_gram_apply": (ctypes.c_int, [_P, _P, _P]),
    "spirec_objective_grad": (ctypes.c_int, [_P, _P, _P, _P]),
    "spirec_toeplitz_noalloc": (ctypes.c_int, [_P, _P, _P, _I32, _I32, _P]),
    "spirec_sync": (ctypes.c_int, [_P]),
    "spirec_plan_info": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "spirec_launch_count": (ctypes.c_int, [_P, _P]),
    "spirec_plan_scalars": (ctypes.c_int, [_P, _P, _I32]),
    "spirec_timing": (ctypes.c_int, [_P, _I32]),
    "spirec_timing_read": (ctypes.c_int, [_P, _P, _P]),
    "spirec_batch_solve": (ctypes.c_int, [_P, _I32, _P, _I32, _P, _P]),
    "spirec_server_create": (ctypes.c_int, [_P, ctypes.c_size_t, _I32, _I32]),
    "spirec_server_plan_bytes": (ctypes.c_int, [_I32, _I64, _I32, _P, _P]),
    "spirec_server_submit": (ctypes.c_int, [_P, _P, _P]),
    "spirec_server_wait": (ctypes.c_int, [_P, ctypes.c_uint64, _I32, _P, _P, _P]),
    "spirec_server_stats": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "spirec_server_destroy": (ctypes.c_int, [_P]),
    "spirec_autotune": (ctypes.c_int, [_P, _I32, _I32, _P, _P]),
    "spirec_tune_set": (ctypes.c_int, [_I32, _I32, _I32, _I32, _I64, _I32, _I32]),
    "spirec_tune_get": (ctypes.c_int, [_I32, _I32, _I32, _I32, _I64, _I32, _P]),
    "spirec_tune_count": (ctypes.c_int, [_P]),
    "spirec_tune_clear": (ctypes.c_int, []),
    "spirec_tune_save": (ctypes.c_int, [ctypes.c_char_p]),
    "spirec_tune_load": (ctypes.c_int, [ctypes.c_char_p]),
    "spirec_inject_alloc_failure": (ctypes.c_int, [_I64]),
    "spirec_set_wait_limit_ns": (ctypes.c_int, [ctypes.c_uint64]),
    "spirec_inject_wait_stall": (ctypes.c_int, [_I32]),
    "spirec_last_error": (ctypes.c_char_p, []),
    "spirec_version": (ctypes.c_char_p, []),
}

_lib = None


class SpirecError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"spirec status {code}: {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    """Load libspirec.so and declare its signatures.  Raises if it is absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise FileNotFoundError(f"{path} is not built; run paper_0908_3252_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(rc):
    if rc != SPIREC_OK:
        raise SpirecError(rc, load().spirec_last_error().decode())
    return rc


def _host_ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _dev_ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device entry points take contiguous CUDA tensors"
    return ctypes.c_void_p(t.data_ptr())


def _c64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.complex64)
    if n is not None:
        assert a.size == n
    return a


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---- thin wrappers with the C names (status checked, pointers marshalled)

def spirec_last_error() -> str:
    return load().spirec_last_error().decode()


def spirec_version() -> str:
    return load().spirec_version().decode()


def spirec_inject_alloc_failure(n):
    """Plan allocations succeed n more times, then fail (n < 0: off)."""
    return _check(load().spirec_inject_alloc_failure(int(n)))


SPIREC_STALL_LOOP = 1
SPIREC_STALL_CONTRACTION = 2


def spirec_inject_wait_stall(kernels):
    """Later launches of the kernels in the mask stall until their wait runs out (0: off)."""
    return _check(load().spirec_inject_wait_stall(int(kernels)))


def spirec_set_wait_limit_ns(ns):
    """Limit of every bounded device wait of later launches (0: the 2 s default)."""
    return _check(load().spirec_set_wait_limit_ns(int(ns)))


def spirec_plan_create(N, L, M=0, precision=SPIREC_FP32, stream=None, kx=None, ky=None):
    plan = ctypes.c_void_p()
    kx = _f64(kx) if kx is not None else None
    ky = _f64(ky) if ky is not None else None
    _check(load().spirec_plan_create(ctypes.byref(plan), int(N), int(L), int(M), int(precision),
                                     ctypes.c_void_p(stream) if stream else None,
                                     _host_ptr(kx), _host_ptr(ky)))
    return plan


def spirec_plan_destroy(plan):
    return _check(load().spirec_plan_destroy(plan))


def spirec_set_trajectory(plan, kx, ky):
    kx, ky = _f64(kx), _f64(ky)
    return _check(load().spirec_set_trajectory(plan, _host_ptr(kx), _host_ptr(ky)))


def spirec_set_trajectory_dev(plan, kx, ky):
    return _check(load().spirec_set_trajectory_dev(plan, _dev_ptr(kx), _dev_ptr(ky)))


def spirec_set_data(plan, s):
    s = _c64(s)
    return _check(load().spirec_set_data(plan, _host_ptr(s)))


def spirec_set_data_dev(plan, s):
    return _check(load().spirec_set_data_dev(plan, _dev_ptr(s)))


def spirec_set_reg(plan, lambda1, alpha1, lambda0, alpha0, phi):
    return _check(load().spirec_set_reg(plan, float(lambda1), float(alpha1), float(lambda0),
                                        float(alpha0), int(phi)))


def spirec_kcache_create(N, M, precision, offsets, kx, ky, stream=None):
    """Per-interleave kernel cache: offsets (n + 1 sample offsets into kx, ky)."""
    off = np.ascontiguousarray(offsets, np.int64)
    kx = np.ascontiguousarray(kx, np.float64)
    ky = np.ascontiguousarray(ky, np.float64)
    h = _P()
    _check(load().spirec_kcache_create(ctypes.byref(h), int(N), int(M), int(precision), int(off.shape[0] - 1),
                                       _host_ptr(off), _host_ptr(kx), _host_ptr(ky), stream))
    return h


def spirec_kcache_destroy(cache):
    return _check(load().spirec_kcache_destroy(cache))


def spirec_set_trajectory_cached(plan, cache, which):
    w = np.ascontiguousarray(which, np.int32)
    return _check(load().spirec_set_trajectory_cached(plan, cache, _host_ptr(w), int(w.shape[0])))


def spirec_set_mode(plan, mode):
    return _check(load().spirec_set_mode(plan, int(mode)))


def spirec_autotune(plan, objective=SPIREC_TUNE_LATENCY, loop_iters=10):
    """Returns (chosen values, median ms of the winners), one per knob."""
    chosen = np.zeros(SPIREC_NUM_KNOBS, np.int32)
    ms = np.zeros(SPIREC_NUM_KNOBS, np.float64)
    _check(load().spirec_autotune(plan, int(objective), int(loop_iters), _host_ptr(chosen), _host_ptr(ms)))
    return chosen, ms


def spirec_tune_set(knob, N, M, precision, L, value, sms=0):
    return _check(load().spirec_tune_set(int(knob), int(N), int(M), int(precision), int(L), int(sms), int(value)))


def spirec_tune_get(knob, N, M, precision, L, sms=0):
    v = ctypes.c_int32(0)
    _check(load().spirec_tune_get(int(knob), int(N), int(M), int(precision), int(L), int(sms), ctypes.byref(v)))
    return v.value


def spirec_tune_count():
    c = ctypes.c_int64(0)
    _check(load().spirec_tune_count(ctypes.byref(c)))
    return c.value


def spirec_tune_clear():
    return _check(load().spirec_tune_clear())


def spirec_tune_save(path):
    return _check(load().spirec_tune_save(os.fsencode(path)))


def spirec_tune_load(path):
    return _check(load().spirec_tune_load(os.fsencode(path)))


def spirec_set_minimiser(plan, kind, inner_iters=0):
    return _check(load().spirec_set_minimiser(plan, int(kind), int(inner_iters)))


def spirec_solve(plan, x0, iters, N):
    """Host variant: returns (x (N,N) complex64, J_hist (iters+1,) float64)."""
    x0 = _c64(x0, N * N) if x0 is not None else None
    x = np.zeros((N, N), np.complex64)
    J = np.zeros(iters + 1, np.float64)
    _check(load().spirec_solve(plan, _host_ptr(x0), int(iters), _host_ptr(x), _host_ptr(J)))
    return x, J


def spirec_solve_dev(plan, x0, iters, x_out, J_hist=None):
    return _check(load().spirec_solve_dev(plan, _dev_ptr(x0), int(iters), _dev_ptr(x_out), _dev_ptr(J_hist)))


def spirec_forward_dev(plan, x, y):
    return _check(load().spirec_forward_dev(plan, _dev_ptr(x), _dev_ptr(y)))


def spirec_adjoint_dev(plan, y, x):
    return _check(load().spirec_adjoint_dev(plan, _dev_ptr(y), _dev_ptr(x)))


def spirec_gram_dev(plan, G):
    return _check(load().spirec_gram_dev(plan, _dev_ptr(G)))


def spirec_kernel_spectrum_dev(plan, C):
    return _check(load().spirec_kernel_spectrum_dev(plan, _dev_ptr(C)))


def spirec_data_adjoint_dev(plan, D):
    return _check(load().spirec_data_adjoint_dev(plan, _dev_ptr(D)))


def spirec_toeplitz_dev(plan, x, Tx):
    return _check(load().spirec_toeplitz_dev(plan, _dev_ptr(x), _dev_ptr(Tx)))


def spirec_objective_grad_dev(plan, x, g):
    J = ctypes.c_double(0.0)
    _check(load().spirec_objective_grad_dev(plan, _dev_ptr(x), ctypes.byref(J), _dev_ptr(g)))
    return J.value


def _plan_sizes(plan):
    N, L = ctypes.c_int32(), ctypes.c_int64()
    _check(load().spirec_plan_info(plan, ctypes.byref(N), ctypes.byref(L), None, None, None))
    return N.value, L.value


def spirec_forward(plan, x):
    """y = H x through host memory: x (N, N) complex64 -> y (L,) complex64."""
    N, L = _plan_sizes(plan)
    x = _c64(x, N * N)
    y = np.empty(L, np.complex64)
    _check(load().spirec_forward(plan, _host_ptr(x), _host_ptr(y)))
    return y


def spirec_adjoint(plan, y):
    """x = H^H y through host memory: y (L,) complex64 -> x (N, N) complex64."""
    N, L = _plan_sizes(plan)
    y = _c64(y, L)
    x = np.empty((N, N), np.complex64)
    _check(load().spirec_adjoint(plan, _host_ptr(y), _host_ptr(x)))
    return x


def spirec_gram_apply(plan, x):
    """T x = H^H H x (zero-padded FFT convolution) through host memory."""
    N, _ = _plan_sizes(plan)
    x = _c64(x, N * N)
    Tx = np.empty((N, N), np.complex64)
    _check(load().spirec_gram_apply(plan, _host_ptr(x), _host_ptr(Tx)))
    return Tx


def spirec_objective_grad(plan, x):
    """(J, g) at x through host memory."""
    N, _ = _plan_sizes(plan)
    x = _c64(x, N * N)
    g = np.empty((N, N), np.complex64)
    J = ctypes.c_double()
    _check(load().spirec_objective_grad(plan, _host_ptr(x), ctypes.byref(J), _host_ptr(g)))
    return J.value, g


def spirec_toeplitz_noalloc(x, spectrum, Tx, N, M, stream=None):
    """T x with no allocation (device tensors; see include/spirec.h)."""
    return _check(load().spirec_toeplitz_noalloc(_dev_ptr(x), _dev_ptr(spectrum), _dev_ptr(Tx), int(N), int(M),
                                                 ctypes.c_void_p(stream) if stream else None))


def spirec_sync(plan):
    return _check(load().spirec_sync(plan))


def spirec_plan_info(plan):
    N, L, M, prec, nbytes = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_size_t()
    _check(load().spirec_plan_info(plan, ctypes.byref(N), ctypes.byref(L), ctypes.byref(M),
                                   ctypes.byref(prec), ctypes.byref(nbytes)))
    return dict(N=N.value, L=L.value, M=M.value, precision=prec.value, device_bytes=nbytes.value)


def spirec_plan_scalars(plan, n=32):
    out = (ctypes.c_double * n)()
    _check(load().spirec_plan_scalars(plan, out, n))
    return list(out)


def spirec_launch_count(plan):
    c = ctypes.c_int64()
    _check(load().spirec_launch_count(plan, ctypes.byref(c)))
    return c.value


def spirec_timing(plan, enable):
    return _check(load().spirec_timing(plan, int(enable)))


def spirec_timing_read(plan):
    ms = (ctypes.c_double * SPIREC_NUM_STAGES)()
    cnt = (ctypes.c_int64 * SPIREC_NUM_STAGES)()
    _check(load().spirec_timing_read(plan, ms, cnt))
    return {STAGES[i]: (ms[i], cnt[i]) for i in range(SPIREC_NUM_STAGES)}


class SpirecRequest(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("L", ctypes.c_int64), ("kx", ctypes.c_void_p), ("ky", ctypes.c_void_p),
                ("s", ctypes.c_void_p), ("lambda1", ctypes.c_double), ("alpha1", ctypes.c_double),
                ("lambda0", ctypes.c_double), ("alpha0", ctypes.c_double), ("phi", ctypes.c_int32),
                ("iters", ctypes.c_int32)]


def spirec_batch_solve(plans, x_out, iters, x0=None, J_hist=None):
    """plans: list of handles; x_out/x0/J_hist: lists of CUDA tensors."""
    n = len(plans)
    P = (ctypes.c_void_p * n)(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in plans])
    X = (ctypes.c_void_p * n)(*[t.data_ptr() for t in x_out])
    X0 = (ctypes.c_void_p * n)(*[t.data_ptr() for t in x0]) if x0 is not None else None
    JH = (ctypes.c_void_p * n)(*[t.data_ptr() for t in J_hist]) if J_hist is not None else None
    return _check(load().spirec_batch_solve(P, n, X0, int(iters), X, JH))


def spirec_server_create(hbm_budget_bytes, max_slots, precision):
    srv = ctypes.c_void_p()
    _check(load().spirec_server_create(ctypes.byref(srv), int(hbm_budget_bytes), int(max_slots), int(precision)))
    return srv


def spirec_server_plan_bytes(N, L, precision):
    """(bytes, M): the request loop's device footprint for a request of this shape."""
    b, m = ctypes.c_size_t(), ctypes.c_int32()
    _check(load().spirec_server_plan_bytes(int(N), int(L), int(precision), ctypes.byref(b), ctypes.byref(m)))
    return b.value, m.value


def spirec_server_submit(srv, N, kx, ky, s, lambda1, alpha1, lambda0, alpha0, phi, iters):
    kx, ky, s = _f64(kx), _f64(ky), _c64(s)
    req = SpirecRequest(int(N), kx.shape[0], kx.ctypes.data, ky.ctypes.data, s.ctypes.data, float(lambda1),
                        float(alpha1), float(lambda0), float(alpha0), int(phi), int(iters))
    t = ctypes.c_uint64()
    _check(load().spirec_server_submit(srv, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def spirec_server_wait(srv, ticket, N, timeout_ms=60000):
    """Returns (x (N,N) complex64, J, latency_s)."""
    x = np.zeros((N, N), np.complex64)
    J, lat = ctypes.c_double(), ctypes.c_double()
    _check(load().spirec_server_wait(srv, ctypes.c_uint64(ticket), int(timeout_ms), _host_ptr(x),
                                     ctypes.byref(J), ctypes.byref(lat)))
    return x, J.value, lat.value


def spirec_server_stats(srv):
    p50, p99 = ctypes.c_double(), ctypes.c_double()
    c, f, q = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().spirec_server_stats(srv, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(c),
                                      ctypes.byref(f), ctypes.byref(q)))
    return dict(p50_s=p50.value, p99_s=p99.value, completed=c.value, failed=f.value, queued=q.value)


def spirec_server_destroy(srv):
    return _check(load().spirec_server_destroy(srv))


# ---- small convenience owner used by the tests and the benchmark

class Plan:
    """Owns a spirec_plan handle; every method is one C-ABI call."""

    def __init__(self, N, L, M=0, precision=SPIREC_FP32, stream=None, kx=None, ky=None):
        self.N, self.L = int(N), int(L)
        self.h = spirec_plan_create(N, L, M, precision, stream, kx, ky)
        self.info = spirec_plan_info(self.h)
        self.M = self.info["M"]

    def close(self):
        if self.h is not None:
            spirec_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
