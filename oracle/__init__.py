"""FP64 CPU oracle for entropic-OT device association (arXiv 1805.01559).

TEST INFRASTRUCTURE ONLY: the test-suite, the package entry point's smoke check
and the benchmark's CPU-baseline leg are the only callers.  The product path
never imports this package.  The arithmetic lives in ``ot_oracle.c`` (plain C,
double precision, loops written to be read against the paper); this module only
compiles it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ot_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, OpenMP, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        pi32 = ctypes.POINTER(ctypes.c_int32)
        lib.oracle_rates.argtypes = [d, d, i64, i64, ctypes.c_double, ctypes.c_double, d]
        lib.oracle_rates_total.argtypes = [d, d, i64, i64, ctypes.c_double, ctypes.c_double, d]
        lib.oracle_cost.argtypes = [d, i64, ctypes.c_double, d]
        lib.oracle_median.argtypes = [d, i64, d]
        lib.oracle_sinkhorn.argtypes = [d, d, d, i64, i64, ctypes.c_double, ctypes.c_double, i32,
                                        d, d, d, pi32, d]
        lib.oracle_plan.argtypes = [d, d, d, i64, i64, ctypes.c_double, d]
        lib.oracle_finalize.argtypes = [d, d, d, d, d, i64, i64, ctypes.c_double, d, d, d, d]
        lib.oracle_maxsinr.argtypes = [d, d, d, i64, i64, pi32, d, d]
        lib.oracle_adaptive.argtypes = [d, d, i64, i64, ctypes.c_double, ctypes.c_double, i32, i32,
                                        ctypes.c_double, d, d, d, d, pi32, d]
        lib.oracle_completion.argtypes = [d, d, d, i64, i64, d, d]
        lib.oracle_euclid_cost.argtypes = [d, d, i64, i64, d]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        for name in ("oracle_rates", "oracle_rates_total", "oracle_cost", "oracle_median", "oracle_sinkhorn",
                     "oracle_plan", "oracle_finalize", "oracle_maxsinr", "oracle_adaptive",
                     "oracle_completion", "oracle_euclid_cost"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"{what}: oracle status {rc}")


def num_threads() -> int:
    return _load().oracle_num_threads()


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def rates(G, P, N0: float, W_hz: float) -> np.ndarray:
    """R_ij = W log2(1 + SINR_ji), Sec. II-A (all other RRHs interfere)."""
    G, P = _f64(G), _f64(P)
    I, J = G.shape
    R = np.empty((I, J))
    _check(_load().oracle_rates(_dp(G), _dp(P), I, J, float(N0), float(W_hz), _dp(R)), "rates")
    return R


def rates_total(G, P, N0: float, W_hz: float) -> np.ndarray:
    """rates() with the interference as row total minus own term (O(I J)), Sec. II-A."""
    G, P = _f64(G), _f64(P)
    I, J = G.shape
    R = np.empty((I, J))
    _check(_load().oracle_rates_total(_dp(G), _dp(P), I, J, float(N0), float(W_hz), _dp(R)), "rates_total")
    return R


def cost(R, mu: float) -> np.ndarray:
    """C_ij = 1 / (mu R_ij), Sec. IV choice (ii)."""
    R = _f64(R)
    C = np.empty_like(R)
    _check(_load().oracle_cost(_dp(R), R.size, float(mu), _dp(C)), "cost")
    return C


def median(x) -> float:
    x = _f64(x).ravel()
    out = np.zeros(1)
    _check(_load().oracle_median(_dp(x), x.size, _dp(out)), "median")
    return float(out[0])


def sinkhorn(C, p, q, eps: float, tol: float, max_iter: int, g0=None):
    """Algorithm 1 in log domain, FP64.  Returns (f, g, iters, row_residual)."""
    C, p, q = _f64(C), _f64(p), _f64(q)
    I, J = C.shape
    f = np.empty(I)
    g = np.empty(J)
    it = ctypes.c_int32(0)
    err = ctypes.c_double(0.0)
    g0keep = _f64(g0) if g0 is not None else None
    g0p = _dp(g0keep) if g0keep is not None else ctypes.POINTER(ctypes.c_double)()
    _check(_load().oracle_sinkhorn(_dp(C), _dp(p), _dp(q), I, J, float(eps), float(tol),
                                   int(max_iter), g0p, _dp(f), _dp(g), ctypes.byref(it),
                                   ctypes.byref(err)), "sinkhorn")
    return f, g, int(it.value), float(err.value)


def plan(C, f, g, eps: float) -> np.ndarray:
    C, f, g = _f64(C), _f64(f), _f64(g)
    I, J = C.shape
    P = np.empty((I, J))
    _check(_load().oracle_plan(_dp(C), _dp(f), _dp(g), I, J, float(eps), _dp(P)), "plan")
    return P


def finalize(C, f, g, p, q, eps: float):
    """(transport cost, rho (J), row L1 error, column L1 error) of the plan (f, g)."""
    C, f, g, p, q = _f64(C), _f64(f), _f64(g), _f64(p), _f64(q)
    I, J = C.shape
    cost_ = ctypes.c_double(0.0)
    er = ctypes.c_double(0.0)
    ec = ctypes.c_double(0.0)
    rho = np.empty(J)
    _check(_load().oracle_finalize(_dp(C), _dp(f), _dp(g), _dp(p), _dp(q), I, J, float(eps),
                                   ctypes.cast(ctypes.byref(cost_), ctypes.POINTER(ctypes.c_double)),
                                   _dp(rho),
                                   ctypes.cast(ctypes.byref(er), ctypes.POINTER(ctypes.c_double)),
                                   ctypes.cast(ctypes.byref(ec), ctypes.POINTER(ctypes.c_double))),
           "finalize")
    return float(cost_.value), rho, float(er.value), float(ec.value)


def maxsinr(R, C, lam):
    """maxSINR association: (assoc (I,), Lambda (J,), total load)."""
    R, C, lam = _f64(R), _f64(C), _f64(lam)
    I, J = R.shape
    assoc = np.empty(I, dtype=np.int32)
    Lam = np.empty(J)
    tot = ctypes.c_double(0.0)
    _check(_load().oracle_maxsinr(_dp(R), _dp(C), _dp(lam), I, J,
                                  assoc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(Lam),
                                  ctypes.cast(ctypes.byref(tot), ctypes.POINTER(ctypes.c_double))),
           "maxsinr")
    return assoc, Lam, float(tot.value)


def adaptive(C, lam, eps: float, tol: float, max_iter: int, outer: int, delta: float):
    """Algorithm 2: (f, g, q used by the last solve, per-step max load)."""
    f, g, q, ml, _, _ = adaptive_trace(C, lam, eps, tol, max_iter, outer, delta)
    return f, g, q, ml


def adaptive_trace(C, lam, eps: float, tol: float, max_iter: int, outer: int, delta: float):
    """Algorithm 2 with its trace: (f, g, q, per-step max load, per-step j*, per-step loads (outer x J))."""
    C, lam = _f64(C), _f64(lam)
    I, J = C.shape
    f = np.empty(I)
    g = np.empty(J)
    q = np.empty(J)
    ml = np.empty(outer)
    js = np.empty(outer, dtype=np.int32)
    rho = np.empty((outer, J))
    _check(_load().oracle_adaptive(_dp(C), _dp(lam), I, J, float(eps), float(tol), int(max_iter),
                                   int(outer), float(delta), _dp(f), _dp(g), _dp(q), _dp(ml),
                                   js.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(rho)),
           "adaptive")
    return f, g, q, ml, js, rho


def completion_time(C, x, lam):
    """Average job completion time of the mass plan x under load costs C, Sec. II-B: (T, rho)."""
    C, x, lam = _f64(C), _f64(x), _f64(lam)
    I, J = C.shape
    T = np.empty(1)
    rho = np.empty(J)
    _check(_load().oracle_completion(_dp(C), _dp(x), _dp(lam), I, J, _dp(T), _dp(rho)), "completion")
    return float(T[0]), rho


def euclid_cost(dev_xy, rrh_xy) -> np.ndarray:
    """C_ij = ||x_i - x_j||, Sec. IV choice (i)."""
    d, r = _f64(dev_xy), _f64(rrh_xy)
    I, J = d.shape[0], r.shape[0]
    C = np.empty((I, J))
    _check(_load().oracle_euclid_cost(_dp(d), _dp(r), I, J, _dp(C)), "euclid_cost")
    return C
