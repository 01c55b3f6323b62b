"""Thin ctypes binding of libot_assoc.so (include/ot_assoc.h), same names as the C ABI.

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels.  PyTorch supplies device memory and the current stream.  There is no CPU
fallback: if the library cannot be loaded, importing ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional

import torch

from . import build as _build

OT_OK = 0
OT_NOT_CONVERGED = 1
OT_EINVAL = -1
OT_ENOMEM = -2
OT_ECUDA = -3
OT_ETIMEOUT = -4
OT_EBUSY = -5
OT_EUNSUPPORTED = -6

OT_KERNEL_F32 = 0
OT_KERNEL_BF16 = 1
OT_KERNEL_F16 = 2

_lib = None


class OTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


def _status_name(s: int) -> str:
    return {0: "OT_OK", 1: "OT_NOT_CONVERGED", -1: "OT_EINVAL", -2: "OT_ENOMEM", -3: "OT_ECUDA",
            -4: "OT_ETIMEOUT", -5: "OT_EBUSY", -6: "OT_EUNSUPPORTED"}.get(s, f"status {s}")


class ot_assoc_result(ctypes.Structure):
    _fields_ = [
        ("pi", ctypes.c_void_p),
        ("pi_ld", ctypes.c_int64),
        ("f", ctypes.c_void_p),
        ("g", ctypes.c_void_p),
        ("rrh_load", ctypes.c_void_p),
        ("transport_cost", ctypes.c_double),
        ("marg_err_row", ctypes.c_double),
        ("marg_err_col", ctypes.c_double),
        ("iters", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("absorptions", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class ot_assoc_timings(ctypes.Structure):
    _fields_ = [
        ("init_ms", ctypes.c_double),
        ("loop_ms", ctypes.c_double),
        ("finalize_ms", ctypes.c_double),
        ("sweeps", ctypes.c_int32),
        ("valid", ctypes.c_int32),
    ]


class ot_assoc_instance(ctypes.Structure):
    _fields_ = [
        ("C", ctypes.c_void_p),
        ("ld", ctypes.c_int64),
        ("I", ctypes.c_int64),
        ("J", ctypes.c_int32),
        ("warm_start", ctypes.c_int32),
        ("p", ctypes.c_void_p),
        ("q", ctypes.c_void_p),
        ("eps", ctypes.c_double),
        ("tol", ctypes.c_double),
        ("max_iter", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("f", ctypes.c_void_p),
        ("g", ctypes.c_void_p),
        ("rrh_load", ctypes.c_void_p),
        ("pi", ctypes.c_void_p),
        ("pi_ld", ctypes.c_int64),
    ]


class ot_assoc_instance_result(ctypes.Structure):
    _fields_ = [
        ("transport_cost", ctypes.c_double),
        ("marg_err_row", ctypes.c_double),
        ("marg_err_col", ctypes.c_double),
        ("err_loop", ctypes.c_double),
        ("iters", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("converged", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


OT_BATCH_NO_GRAPH = 1

# (name, restype, argtypes) of every exported entry point in include/ot_assoc.h
_VP, _I64, _I32, _D, _SZ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_size_t
_PD = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "ot_assoc_version": (ctypes.c_int, []),
    "ot_assoc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ot_assoc_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, _SZ]),
    "ot_assoc_destroy": (None, [_VP]),
    "ot_assoc_last_error": (ctypes.c_char_p, [_VP]),
    "ot_assoc_scratch_bytes": (_SZ, [_VP]),
    "ot_assoc_set_spin_limit": (None, [_VP, _I64]),
    "ot_assoc_enable_timing": (None, [_VP, ctypes.c_int]),
    "ot_assoc_last_timings": (ctypes.c_int, [_VP, ctypes.POINTER(ot_assoc_timings)]),
    "ot_assoc_launch_count": (ctypes.c_uint64, [_VP]),
    "ot_assoc_build_rates": (ctypes.c_int, [_VP, _VP, _I64, _VP, _I64, _I64, _D, _D, _VP, _I64, _VP]),
    "ot_assoc_build_cost": (ctypes.c_int, [_VP, _VP, _I64, _I64, _I64, _D, _VP, _I64, _D, _PD, _VP]),
    "ot_assoc_median_f32": (ctypes.c_int, [_VP, _VP, _I64, _PD, _VP]),
    "ot_assoc_maxsinr": (ctypes.c_int, [_VP, _VP, _I64, _VP, _I64, _I64, _D, _VP, _VP, _PD, _VP]),
    "ot_assoc_solve": (ctypes.c_int, [_VP, _VP, _I64, _VP, _VP, _I64, _I64, _D, _D, _D, _I32, _I32,
                                      ctypes.POINTER(ot_assoc_result), _VP]),
    "ot_assoc_solve_cost": (ctypes.c_int, [_VP, _VP, _I64, _VP, _VP, _I64, _I64, _D, _D, _I32, _I32,
                                           ctypes.POINTER(ot_assoc_result), _VP]),
    "ot_assoc_solve_cost_noalloc": (ctypes.c_int, [_VP, _I64, _VP, _VP, _I64, _I64, _D, _D, _I32, _I32,
                                                   ctypes.POINTER(ot_assoc_result), _VP]),
    "ot_assoc_solve_f64": (ctypes.c_int, [_VP, _VP, _I64, _VP, _VP, _I64, _I64, _D, _D, _I32, _I32,
                                          ctypes.POINTER(ot_assoc_result), _VP]),
    "ot_assoc_solve_lowp": (ctypes.c_int, [_VP, _VP, _I64, _VP, _VP, _I64, _I64, _D, _D, _I32, _I32,
                                           _I32, _D, ctypes.POINTER(ot_assoc_result), _VP]),
    "ot_assoc_solve_batched": (ctypes.c_int, [_VP, ctypes.POINTER(ot_assoc_instance), _I32,
                                              ctypes.POINTER(ot_assoc_instance_result), _VP]),
    "ot_assoc_batch_create": (ctypes.c_int, [_VP, ctypes.POINTER(ot_assoc_instance), _I32, _I32,
                                             ctypes.POINTER(_VP)]),
    "ot_assoc_batch_set": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(ot_assoc_instance)]),
    "ot_assoc_batch_launch": (ctypes.c_int, [_VP, _VP]),
    "ot_assoc_batch_wait": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ot_assoc_instance_result)]),
    "ot_assoc_batch_destroy": (None, [_VP]),
    "ot_assoc_autotune": (ctypes.c_int, [_VP, ctypes.POINTER(ot_assoc_instance), _I32, _I32, _VP]),
    "ot_assoc_tuning_get": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32), _PD]),
    "ot_assoc_tuning_set": (ctypes.c_int, [_VP, _I32, _I32, _I32]),
    "ot_assoc_bucket": (_I32, [_I64, _I32]),
}


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libot_assoc.so (building it first if asked).  Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError(f"{path} is missing: run paper_1805_01559_gb300.build.build()")
        _build.build()
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _need(t: torch.Tensor, dtype, name: str, dims: int):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.dim() != dims:
        raise ValueError(f"{name} must have {dims} dims")
    if dims == 2:
        if t.stride(1) != 1:
            raise ValueError(f"{name} must be row-major with unit column stride")
    elif not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


@dataclasses.dataclass
class Result:
    f: torch.Tensor
    g: torch.Tensor
    pi: Optional[torch.Tensor]
    rrh_load: Optional[torch.Tensor]
    transport_cost: float
    marg_err_row: float
    marg_err_col: float
    iters: int
    status: int
    absorptions: int

    @property
    def converged(self) -> bool:
        return self.status == OT_OK


class Context:
    """One library context (scratch arena) on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self._L = lib()
        h = ctypes.c_void_p()
        st = self._L.ot_assoc_create(ctypes.byref(h), int(device), int(hbm_budget_bytes))
        if st != OT_OK:
            raise OTError(st, "ot_assoc_create failed")
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            self._L.ot_assoc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    def last_error(self) -> str:
        return self._L.ot_assoc_last_error(self._h).decode()

    def scratch_bytes(self) -> int:
        return int(self._L.ot_assoc_scratch_bytes(self._h))

    def set_spin_limit(self, polls: int) -> None:
        self._L.ot_assoc_set_spin_limit(self._h, int(polls))

    def enable_timing(self, on: bool = True) -> None:
        self._L.ot_assoc_enable_timing(self._h, 1 if on else 0)

    def last_timings(self) -> dict:
        t = ot_assoc_timings()
        self._L.ot_assoc_last_timings(self._h, ctypes.byref(t))
        return {"init_ms": t.init_ms, "loop_ms": t.loop_ms, "finalize_ms": t.finalize_ms,
                "sweeps": t.sweeps, "valid": bool(t.valid)}

    def launch_count(self) -> int:
        return int(self._L.ot_assoc_launch_count(self._h))

    def _check(self, st: int, allow_nc: bool = False) -> int:
        if st == OT_OK or (allow_nc and st == OT_NOT_CONVERGED):
            return st
        raise OTError(st, self.last_error())

    # ---- cost construction --------------------------------------------------------------
    def build_rates(self, G: torch.Tensor, P: torch.Tensor, N0: float, W_hz: float,
                    R_out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        _need(G, torch.float32, "G", 2)
        _need(P, torch.float32, "P", 1)
        I, J = G.shape
        if R_out is None:
            R_out = torch.empty((I, J), dtype=torch.float32, device=G.device)
        self._check(self._L.ot_assoc_build_rates(self._h, _ptr(G), G.stride(0), _ptr(P), I, J, float(N0),
                                                 float(W_hz), _ptr(R_out), R_out.stride(0), _stream(stream)))
        return R_out

    def build_cost(self, R: torch.Tensor, mu: float, eps_rel: Optional[float] = None,
                   C_out: Optional[torch.Tensor] = None, stream=None):
        _need(R, torch.float32, "R", 2)
        I, J = R.shape
        if C_out is None:
            C_out = torch.empty((I, J), dtype=torch.float32, device=R.device)
        eps = ctypes.c_double(0.0)
        self._check(self._L.ot_assoc_build_cost(self._h, _ptr(R), R.stride(0), I, J, float(mu), _ptr(C_out),
                                                C_out.stride(0), float(eps_rel or 0.0),
                                                ctypes.byref(eps) if eps_rel is not None else None,
                                                _stream(stream)))
        return C_out, (eps.value if eps_rel is not None else None)

    def median_f32(self, x: torch.Tensor, stream=None) -> float:
        _need(x, torch.float32, "x", 1)
        out = ctypes.c_double(0.0)
        self._check(self._L.ot_assoc_median_f32(self._h, _ptr(x), x.numel(), ctypes.byref(out), _stream(stream)))
        return out.value

    def maxsinr(self, R: torch.Tensor, traffic: torch.Tensor, mu: float, stream=None):
        _need(R, torch.float32, "R", 2)
        _need(traffic, torch.float32, "traffic", 1)
        I, J = R.shape
        assoc = torch.empty(I, dtype=torch.int32, device=R.device)
        Lam = torch.empty(J, dtype=torch.float64, device=R.device)
        tot = ctypes.c_double(0.0)
        self._check(self._L.ot_assoc_maxsinr(self._h, _ptr(R), R.stride(0), _ptr(traffic), I, J, float(mu),
                                             _ptr(assoc), _ptr(Lam), ctypes.byref(tot), _stream(stream)))
        return assoc, Lam, tot.value

    # ---- solves -------------------------------------------------------------------------
    def _result(self, I, J, device, want_pi, want_load, f, g):
        f = torch.empty(I, dtype=torch.float64, device=device) if f is None else f
        g = torch.empty(J, dtype=torch.float64, device=device) if g is None else g
        pi = torch.empty((I, J), dtype=torch.float32, device=device) if want_pi else None
        load = torch.empty(J, dtype=torch.float64, device=device) if want_load else None
        r = ot_assoc_result()
        r.pi = pi.data_ptr() if pi is not None else None
        r.pi_ld = J
        r.f = f.data_ptr()
        r.g = g.data_ptr()
        r.rrh_load = load.data_ptr() if load is not None else None
        return r, f, g, pi, load

    @staticmethod
    def _pack(r, f, g, pi, load) -> Result:
        return Result(f=f, g=g, pi=pi, rrh_load=load, transport_cost=r.transport_cost,
                      marg_err_row=r.marg_err_row, marg_err_col=r.marg_err_col, iters=r.iters,
                      status=r.status, absorptions=r.absorptions)

    def solve(self, R, traffic, rrh_marginal, mu, eps, tol=1e-6, max_iter=2000, warm_g=None,
              want_pi=False, want_load=True, f=None, g=None, stream=None) -> Result:
        """Algorithm 1 on C = 1/(mu R) (FP32 log domain).  warm_g: start from b = exp(g/eps)."""
        _need(R, torch.float32, "R", 2)
        _need(traffic, torch.float32, "traffic", 1)
        _need(rrh_marginal, torch.float32, "rrh_marginal", 1)
        I, J = R.shape
        if warm_g is not None:
            g = warm_g if g is None else g.copy_(warm_g)
        r, f, g, pi, load = self._result(I, J, R.device, want_pi, want_load, f, g)
        st = self._L.ot_assoc_solve(self._h, _ptr(R), R.stride(0), _ptr(traffic), _ptr(rrh_marginal), I, J,
                                    float(mu), float(eps), float(tol), int(max_iter), int(warm_g is not None),
                                    ctypes.byref(r), _stream(stream))
        self._check(st, allow_nc=True)
        return self._pack(r, f, g, pi, load)

    def solve_cost(self, C, p, q, eps, tol=1e-6, max_iter=2000, warm_g=None, want_pi=False,
                   want_load=True, f=None, g=None, stream=None) -> Result:
        _need(C, torch.float32, "C", 2)
        _need(p, torch.float32, "p", 1)
        _need(q, torch.float32, "q", 1)
        I, J = C.shape
        if warm_g is not None:
            g = warm_g if g is None else g.copy_(warm_g)
        r, f, g, pi, load = self._result(I, J, C.device, want_pi, want_load, f, g)
        st = self._L.ot_assoc_solve_cost(self._h, _ptr(C), C.stride(0), _ptr(p), _ptr(q), I, J, float(eps),
                                         float(tol), int(max_iter), int(warm_g is not None), ctypes.byref(r),
                                         _stream(stream))
        self._check(st, allow_nc=True)
        return self._pack(r, f, g, pi, load)

    def solve_f64(self, C, p, q, eps, tol=1e-6, max_iter=2000, warm_g=None, want_pi=False,
                  want_load=True, stream=None) -> Result:
        _need(C, torch.float64, "C", 2)
        _need(p, torch.float64, "p", 1)
        _need(q, torch.float64, "q", 1)
        I, J = C.shape
        g = warm_g.clone() if warm_g is not None else None
        r, f, g, pi, load = self._result(I, J, C.device, want_pi, want_load, None, g)
        st = self._L.ot_assoc_solve_f64(self._h, _ptr(C), C.stride(0), _ptr(p), _ptr(q), I, J, float(eps),
                                        float(tol), int(max_iter), int(warm_g is not None), ctypes.byref(r),
                                        _stream(stream))
        self._check(st, allow_nc=True)
        return self._pack(r, f, g, pi, load)

    def solve_lowp(self, C, p, q, eps, tol=1e-3, max_iter=2000, fmt=OT_KERNEL_BF16, absorb_log2=0.0,
                   warm_g=None, want_pi=False, want_load=True, stream=None) -> Result:
        _need(C, torch.float32, "C", 2)
        _need(p, torch.float32, "p", 1)
        _need(q, torch.float32, "q", 1)
        I, J = C.shape
        g = warm_g.clone() if warm_g is not None else None
        r, f, g, pi, load = self._result(I, J, C.device, want_pi, want_load, None, g)
        st = self._L.ot_assoc_solve_lowp(self._h, _ptr(C), C.stride(0), _ptr(p), _ptr(q), I, J, float(eps),
                                         float(tol), int(max_iter), int(warm_g is not None), int(fmt),
                                         float(absorb_log2), ctypes.byref(r), _stream(stream))
        self._check(st, allow_nc=True)
        return self._pack(r, f, g, pi, load)


# ---- batched ragged solves ------------------------------------------------------------------
@dataclasses.dataclass
class Instance:
    """One instance of a batch: cost C (I x J, float32, 16-byte aligned rows), marginals, eps.
    f, g (float64) receive the potentials; g is read first when warm_start."""
    C: torch.Tensor
    p: torch.Tensor
    q: torch.Tensor
    eps: float
    tol: float = 1e-6
    max_iter: int = 2000
    warm_start: bool = False
    f: Optional[torch.Tensor] = None
    g: Optional[torch.Tensor] = None
    rrh_load: Optional[torch.Tensor] = None
    pi: Optional[torch.Tensor] = None

    def prepare(self, want_load: bool = True) -> "Instance":
        _need(self.C, torch.float32, "C", 2)
        _need(self.p, torch.float32, "p", 1)
        _need(self.q, torch.float32, "q", 1)
        I, J = self.C.shape
        dev = self.C.device
        if self.f is None:
            self.f = torch.empty(I, dtype=torch.float64, device=dev)
        if self.g is None:
            self.g = torch.zeros(J, dtype=torch.float64, device=dev)
        if want_load and self.rrh_load is None:
            self.rrh_load = torch.empty(J, dtype=torch.float64, device=dev)
        return self

    def to_c(self) -> ot_assoc_instance:
        I, J = self.C.shape
        d = ot_assoc_instance()
        d.C = self.C.data_ptr()
        d.ld = self.C.stride(0)
        d.I = I
        d.J = J
        d.warm_start = 1 if self.warm_start else 0
        d.p = self.p.data_ptr()
        d.q = self.q.data_ptr()
        d.eps = float(self.eps)
        d.tol = float(self.tol)
        d.max_iter = int(self.max_iter)
        d.f = self.f.data_ptr()
        d.g = self.g.data_ptr()
        d.rrh_load = self.rrh_load.data_ptr() if self.rrh_load is not None else None
        d.pi = self.pi.data_ptr() if self.pi is not None else None
        d.pi_ld = self.pi.stride(0) if self.pi is not None else 0
        return d


@dataclasses.dataclass
class InstanceResult:
    transport_cost: float
    marg_err_row: float
    marg_err_col: float
    err_loop: float
    iters: int
    status: int
    converged: bool


def _results(arr, n) -> list:
    return [InstanceResult(arr[k].transport_cost, arr[k].marg_err_row, arr[k].marg_err_col, arr[k].err_loop,
                           arr[k].iters, arr[k].status, bool(arr[k].converged)) for k in range(n)]


class Batch:
    """A planned batch (ot_assoc_batch): schedule, device tables and a captured CUDA graph."""

    def __init__(self, ctx: "Context", instances, graph: bool = True):
        self._ctx = ctx
        self._L = ctx._L
        self.instances = [x.prepare() for x in instances]
        n = len(self.instances)
        arr = (ot_assoc_instance * n)(*[x.to_c() for x in self.instances])
        h = ctypes.c_void_p()
        st = self._L.ot_assoc_batch_create(ctx.handle, arr, n, 0 if graph else OT_BATCH_NO_GRAPH, ctypes.byref(h))
        ctx._check(st)
        self._h = h
        self._res = (ot_assoc_instance_result * n)()

    def set(self, k: int, inst: Instance) -> None:
        inst.prepare()
        d = inst.to_c()
        self._ctx._check(self._L.ot_assoc_batch_set(self._h, int(k), ctypes.byref(d)))
        self.instances[k] = inst

    def launch(self, stream=None) -> None:
        self._ctx._check(self._L.ot_assoc_batch_launch(self._h, _stream(stream)))

    def wait(self, stream=None) -> list:
        self._ctx._check(self._L.ot_assoc_batch_wait(self._h, _stream(stream), self._res))
        return _results(self._res, len(self.instances))

    def run(self, stream=None) -> list:
        self.launch(stream)
        return self.wait(stream)

    def close(self):
        if getattr(self, "_h", None):
            self._L.ot_assoc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ctx_solve_batched(self, instances, stream=None) -> list:
    """One-shot batched solve (ot_assoc_solve_batched); fills each instance's f, g, rrh_load."""
    inst = [x.prepare() for x in instances]
    n = len(inst)
    arr = (ot_assoc_instance * n)(*[x.to_c() for x in inst])
    res = (ot_assoc_instance_result * n)()
    self._check(self._L.ot_assoc_solve_batched(self._h, arr, n, res, _stream(stream)))
    return _results(res, n)


def _ctx_autotune(self, instances, iters: int = 8, stream=None) -> None:
    inst = [x.prepare() for x in instances]
    n = len(inst)
    arr = (ot_assoc_instance * n)(*[x.to_c() for x in inst])
    self._check(self._L.ot_assoc_autotune(self._h, arr, n, int(iters), _stream(stream)))


def _ctx_tuning(self) -> list:
    out = []
    for b in range(15):
        gs, stg, rate = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0.0)
        self._check(self._L.ot_assoc_tuning_get(self._h, b, ctypes.byref(gs), ctypes.byref(stg), ctypes.byref(rate)))
        out.append({"bucket": b, "gsize": gs.value, "stage": stg.value, "rate": rate.value})
    return out


def _ctx_set_tuning(self, bucket: int, gsize: int, stage: int) -> None:
    self._check(self._L.ot_assoc_tuning_set(self._h, int(bucket), int(gsize), int(stage)))


def bucket(I: int, J: int) -> int:
    return int(lib().ot_assoc_bucket(int(I), int(J)))



Context.solve_batched = _ctx_solve_batched
Context.autotune = _ctx_autotune
Context.tuning = _ctx_tuning
Context.set_tuning = _ctx_set_tuning
Context.batch = lambda self, instances, graph=True: Batch(self, instances, graph)


# ---- serving ------------------------------------------------------------------------------
class ot_assoc_server_config(ctypes.Structure):
    _fields_ = [("group_ctas", ctypes.c_int32), ("max_J", ctypes.c_int32), ("idle_us", ctypes.c_double),
                ("hbm_budget", ctypes.c_size_t)]


class ot_assoc_cell_desc(ctypes.Structure):
    _fields_ = [
        ("I", ctypes.c_int64), ("J", ctypes.c_int32), ("warm_start", ctypes.c_int32),
        ("eps", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
        ("reserved", ctypes.c_int32), ("eps_rel", ctypes.c_double), ("mu", ctypes.c_double),
        ("N0", ctypes.c_double), ("W_hz", ctypes.c_double),
        ("P", ctypes.c_void_p), ("p", ctypes.c_void_p), ("q", ctypes.c_void_p),
        ("dev_xy", ctypes.c_void_p), ("dev_v", ctypes.c_void_p), ("rrh_xy", ctypes.c_void_p),
        ("shadow_db", ctypes.c_void_p), ("side_m", ctypes.c_double),
    ]


class ot_assoc_server_result(ctypes.Structure):
    _fields_ = [
        ("ticket", ctypes.c_uint64), ("cell", ctypes.c_int32), ("status", ctypes.c_int32),
        ("iters", ctypes.c_int32), ("reserved", ctypes.c_int32), ("transport_cost", ctypes.c_double),
        ("marg_err_row", ctypes.c_double), ("marg_err_col", ctypes.c_double), ("t_submit_us", ctypes.c_double),
        ("t_start_us", ctypes.c_double), ("t_done_us", ctypes.c_double),
    ]


class ot_assoc_server_stats_t(ctypes.Structure):
    _fields_ = [("resident_bytes", ctypes.c_size_t), ("cells", ctypes.c_int32), ("groups", ctypes.c_int32),
                ("group_ctas", ctypes.c_int32), ("waiting", ctypes.c_int32), ("inflight", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("launches", ctypes.c_uint64)]


SIGNATURES.update({
    "ot_assoc_server_create": (ctypes.c_int, [_VP, ctypes.POINTER(ot_assoc_server_config), ctypes.POINTER(_VP)]),
    "ot_assoc_server_destroy": (None, [_VP]),
    "ot_assoc_server_add_cell": (ctypes.c_int, [_VP, ctypes.POINTER(ot_assoc_cell_desc),
                                                ctypes.POINTER(ctypes.c_int32)]),
    "ot_assoc_server_submit": (ctypes.c_int, [_VP, _I32, _VP, _I64, _D, ctypes.POINTER(ctypes.c_uint64)]),
    "ot_assoc_server_poll": (ctypes.c_int, [_VP, ctypes.POINTER(ot_assoc_server_result), _I32,
                                            ctypes.POINTER(ctypes.c_int32)]),
    "ot_assoc_server_drain": (ctypes.c_int, [_VP, _D]),
    "ot_assoc_server_cell_state": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                                  ctypes.POINTER(_VP), ctypes.POINTER(_VP)]),
    "ot_assoc_server_stats": (ctypes.c_int, [_VP, ctypes.POINTER(ot_assoc_server_stats_t)]),
    "ot_assoc_server_cell_eps": (ctypes.c_int, [_VP, _I32, _PD]),
})
if _lib is not None:  # already loaded: register the new entry points
    for _name in ("ot_assoc_server_create", "ot_assoc_server_destroy", "ot_assoc_server_add_cell",
                  "ot_assoc_server_submit", "ot_assoc_server_poll", "ot_assoc_server_drain",
                  "ot_assoc_server_cell_state", "ot_assoc_server_stats", "ot_assoc_server_cell_eps"):
        _fn = getattr(_lib, _name)
        _fn.restype, _fn.argtypes = SIGNATURES[_name]


@dataclasses.dataclass
class ServerResult:
    ticket: int
    cell: int
    status: int
    iters: int
    transport_cost: float
    marg_err_row: float
    marg_err_col: float
    t_submit_us: float
    t_start_us: float
    t_done_us: float

    @property
    def latency_us(self) -> float:
        return self.t_done_us - self.t_submit_us


class Server:
    """ot_assoc_server: resident cells, continuously batched warm-started solves."""

    def __init__(self, ctx: "Context", group_ctas: int = 0, max_J: int = 1024, idle_us: float = 200.0,
                 hbm_budget: int = 0):
        self._ctx = ctx
        self._L = ctx._L
        cfg = ot_assoc_server_config(int(group_ctas), int(max_J), float(idle_us), int(hbm_budget))
        h = ctypes.c_void_p()
        ctx._check(self._L.ot_assoc_server_create(ctx.handle, ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._keep = {}  # host arrays and request gains kept alive

    def add_cell(self, I, J, eps, P, p, q, mu, N0, W_hz, tol=1e-6, max_iter=2000, warm_start=True,
                 dev_xy=None, dev_v=None, rrh_xy=None, shadow_db=None, side_m=0.0, eps_rel=0.0) -> int:
        """Register a cell; eps <= 0 with eps_rel > 0 (drifting cells) takes eps = eps_rel x
        median(C) of the first instance."""
        import numpy as np
        arrs = {"P": np.ascontiguousarray(P, np.float32), "p": np.ascontiguousarray(p, np.float32),
                "q": np.ascontiguousarray(q, np.float32)}
        if dev_xy is not None:
            arrs.update(dev_xy=np.ascontiguousarray(dev_xy, np.float64), dev_v=np.ascontiguousarray(dev_v, np.float64),
                        rrh_xy=np.ascontiguousarray(rrh_xy, np.float32),
                        shadow_db=np.ascontiguousarray(shadow_db, np.float32))
        d = ot_assoc_cell_desc()
        d.I, d.J, d.warm_start = int(I), int(J), 1 if warm_start else 0
        d.eps, d.tol, d.max_iter, d.eps_rel = float(eps), float(tol), int(max_iter), float(eps_rel)
        d.mu, d.N0, d.W_hz = float(mu), float(N0), float(W_hz)
        for k, v in arrs.items():
            setattr(d, k, v.ctypes.data)
        d.side_m = float(side_m)
        cid = ctypes.c_int32(-1)
        self._ctx._check(self._L.ot_assoc_server_add_cell(self._h, ctypes.byref(d), ctypes.byref(cid)))
        return cid.value

    def cell_eps(self, cell: int) -> float:
        e = ctypes.c_double(0.0)
        self._ctx._check(self._L.ot_assoc_server_cell_eps(self._h, int(cell), ctypes.byref(e)))
        return e.value

    def submit(self, cell: int, G: Optional[torch.Tensor] = None, dt: float = 0.0) -> int:
        t = ctypes.c_uint64(0)
        if G is not None:
            _need(G, torch.float32, "G", 2)
        self._ctx._check(self._L.ot_assoc_server_submit(self._h, int(cell), _ptr(G), G.stride(0) if G is not None else 0,
                                                        float(dt), ctypes.byref(t)))
        if G is not None:
            self._keep[t.value] = G
        return t.value

    def poll(self, max_results: int = 256) -> list:
        arr = (ot_assoc_server_result * max_results)()
        n = ctypes.c_int32(0)
        self._ctx._check(self._L.ot_assoc_server_poll(self._h, arr, int(max_results), ctypes.byref(n)))
        out = []
        for k in range(n.value):
            r = arr[k]
            self._keep.pop(r.ticket, None)
            out.append(ServerResult(r.ticket, r.cell, r.status, r.iters, r.transport_cost, r.marg_err_row,
                                    r.marg_err_col, r.t_submit_us, r.t_start_us, r.t_done_us))
        return out

    def drain(self, timeout_s: float = 60.0) -> list:
        self._ctx._check(self._L.ot_assoc_server_drain(self._h, float(timeout_s)))
        out = []
        while True:
            got = self.poll()
            out += got
            if len(got) == 0:
                return out

    def cell_state(self, cell: int, I: int, J: int):
        """(C, f, g, rho) of a cell: copies of the resident device buffers."""
        C, f, g, rho = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        self._ctx._check(self._L.ot_assoc_server_cell_state(self._h, int(cell), ctypes.byref(C), ctypes.byref(f),
                                                            ctypes.byref(g), ctypes.byref(rho)))
        ldc = (J + 3) // 4 * 4
        torch.cuda.synchronize()
        Cv = _device_view(C.value, (I, ldc), "<f4")[:, :J].clone()
        return (Cv, _device_view(f.value, (I,), "<f8").clone(), _device_view(g.value, (J,), "<f8").clone(),
                _device_view(rho.value, (J,), "<f8").clone())

    def stats(self) -> dict:
        s = ot_assoc_server_stats_t()
        self._ctx._check(self._L.ot_assoc_server_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._L.ot_assoc_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DevBuf:
    """A library-owned device buffer described by the CUDA array interface."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def _device_view(ptr: int, shape, typestr: str) -> torch.Tensor:
    return torch.as_tensor(_DevBuf(ptr, shape, typestr), device="cuda")


Context.server = lambda self, **kw: Server(self, **kw)


# ---- adaptive Sinkhorn association (Algorithm 2) ----------------------------------------------
class ot_assoc_adaptive_params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("tol", ctypes.c_double), ("delta", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("outer", ctypes.c_int32), ("cold_start", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ot_assoc_adaptive_step(ctypes.Structure):
    _fields_ = [("max_load", ctypes.c_double), ("transport_cost", ctypes.c_double),
                ("marg_err_row", ctypes.c_double), ("marg_err_col", ctypes.c_double), ("err_loop", ctypes.c_double),
                ("jstar", ctypes.c_int32), ("iters", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("status", ctypes.c_int32)]


SIGNATURES["ot_assoc_adaptive"] = (ctypes.c_int, [_VP, _VP, _I64, _VP, _I64, _I64,
                                                  ctypes.POINTER(ot_assoc_adaptive_params), _VP, _VP, _VP, _VP,
                                                  _VP, _I64, ctypes.POINTER(ot_assoc_adaptive_step), _VP])
if _lib is not None:
    _lib.ot_assoc_adaptive.restype, _lib.ot_assoc_adaptive.argtypes = SIGNATURES["ot_assoc_adaptive"]


@dataclasses.dataclass
class AdaptiveResult:
    f: torch.Tensor
    g: torch.Tensor
    q: torch.Tensor                    # FP64 targets the last solve used
    rrh_load: torch.Tensor             # rho_j of the last plan
    pi: Optional[torch.Tensor]
    steps: list                        # per outer step: dict(jstar, max_load, iters, ...)
    status: int


def _ctx_adaptive(self, C, traffic, eps, delta, outer, tol=1e-6, max_iter=2000, cold_start=False,
                  want_pi=False, stream=None) -> AdaptiveResult:
    """Algorithm 2: `outer` steps of (solve with q, most loaded RRH j*, move delta off j*)."""
    _need(C, torch.float32, "C", 2)
    _need(traffic, torch.float32, "traffic", 1)
    I, J = C.shape
    dev = C.device
    f = torch.empty(I, dtype=torch.float64, device=dev)
    g = torch.empty(J, dtype=torch.float64, device=dev)
    q = torch.empty(J, dtype=torch.float64, device=dev)
    load = torch.empty(J, dtype=torch.float64, device=dev)
    pi = torch.empty((I, J), dtype=torch.float32, device=dev) if want_pi else None
    prm = ot_assoc_adaptive_params(eps=float(eps), tol=float(tol), delta=float(delta), max_iter=int(max_iter),
                                   outer=int(outer), cold_start=int(bool(cold_start)), reserved=0)
    steps = (ot_assoc_adaptive_step * max(1, int(outer)))()
    st = self._L.ot_assoc_adaptive(self._h, _ptr(C), C.stride(0), _ptr(traffic), I, J, ctypes.byref(prm),
                                   _ptr(f), _ptr(g), _ptr(q), _ptr(load), _ptr(pi), J if want_pi else 0, steps,
                                   _stream(stream))
    self._check(st, allow_nc=True)
    out = [{k: getattr(s, k) for k, _ in ot_assoc_adaptive_step._fields_} for s in steps[:int(outer)]]
    return AdaptiveResult(f=f, g=g, q=q, rrh_load=load, pi=pi, steps=out, status=st)


Context.adaptive = _ctx_adaptive


# ---- policy evaluation: Euclidean cost, completion time (Sec. II-B, Sec. IV) -------------------
SIGNATURES["ot_assoc_euclid_cost"] = (ctypes.c_int, [_VP, _VP, _VP, _I64, _I64, _VP, _I64, _VP])
SIGNATURES["ot_assoc_completion_time"] = (ctypes.c_int, [_VP, _VP, _I64, _VP, _I64, _I64, _VP, _VP, _I64, _VP,
                                                         _VP, _D, _VP, _PD, _VP])
if _lib is not None:
    for _name in ("ot_assoc_euclid_cost", "ot_assoc_completion_time"):
        _fn = getattr(_lib, _name)
        _fn.restype, _fn.argtypes = SIGNATURES[_name]


def _ctx_euclid_cost(self, dev_xy, rrh_xy, C_out=None, stream=None) -> torch.Tensor:
    """C_ij = ||x_i - x_j|| (Sec. IV cost choice (i)); dev_xy I x 2, rrh_xy J x 2 float32."""
    _need(dev_xy, torch.float32, "dev_xy", 2)
    _need(rrh_xy, torch.float32, "rrh_xy", 2)
    if not dev_xy.is_contiguous() or not rrh_xy.is_contiguous() or dev_xy.shape[1] != 2 or rrh_xy.shape[1] != 2:
        raise ValueError("coordinates must be contiguous (n, 2) tensors")
    I, J = dev_xy.shape[0], rrh_xy.shape[0]
    if C_out is None:
        ld = (J + 3) // 4 * 4
        C_out = torch.empty((I, ld), dtype=torch.float32, device=dev_xy.device)[:, :J]
    _need(C_out, torch.float32, "C_out", 2)
    self._check(self._L.ot_assoc_euclid_cost(self._h, _ptr(dev_xy), _ptr(rrh_xy), I, J, _ptr(C_out),
                                             C_out.stride(0), _stream(stream)))
    return C_out


def _ctx_completion_time(self, C, traffic, assoc=None, f=None, g=None, eps=0.0, C_plan=None, want_rho=True,
                         stream=None):
    """Average job completion time (Sec. II-B) of a hard association or of the entropic plan of
    potentials (f, g) on C_plan (default C); C is the load cost.  Returns (T, rho)."""
    _need(C, torch.float32, "C", 2)
    _need(traffic, torch.float32, "traffic", 1)
    I, J = C.shape
    if assoc is not None:
        _need(assoc, torch.int32, "assoc", 1)
    if C_plan is not None:
        _need(C_plan, torch.float32, "C_plan", 2)
    rho = torch.empty(J, dtype=torch.float64, device=C.device) if want_rho else None
    T = ctypes.c_double(0.0)
    self._check(self._L.ot_assoc_completion_time(
        self._h, _ptr(C), C.stride(0), _ptr(traffic), I, J, _ptr(assoc), _ptr(C_plan),
        C_plan.stride(0) if C_plan is not None else 0, _ptr(f), _ptr(g), float(eps), _ptr(rho), ctypes.byref(T),
        _stream(stream)))
    return T.value, rho


Context.euclid_cost = _ctx_euclid_cost
Context.completion_time = _ctx_completion_time


SIGNATURES["ot_assoc_mean_row_min"] = (ctypes.c_int, [_VP, _VP, _I64, _I64, _I64, _PD, _VP])
if _lib is not None:
    _lib.ot_assoc_mean_row_min.restype, _lib.ot_assoc_mean_row_min.argtypes = SIGNATURES["ot_assoc_mean_row_min"]


def _ctx_mean_row_min(self, C, stream=None) -> float:
    """Mean over rows of min_j C_ij (the cost of each device's cheapest link)."""
    _need(C, torch.float32, "C", 2)
    out = ctypes.c_double(0.0)
    self._check(self._L.ot_assoc_mean_row_min(self._h, _ptr(C), C.stride(0), C.shape[0], C.shape[1],
                                              ctypes.byref(out), _stream(stream)))
    return out.value


Context.mean_row_min = _ctx_mean_row_min


# ---- eps-scaling ----------------------------------------------------------------------------------
SIGNATURES["ot_assoc_solve_eps_scaling"] = (ctypes.c_int, [_VP, _VP, _I64, _VP, _VP, _I64, _I64, _D, _D, _D, _D,
                                                           _D, _I32, _I32, ctypes.POINTER(ot_assoc_result),
                                                           ctypes.POINTER(ctypes.c_int32),
                                                           ctypes.POINTER(ctypes.c_int32), _VP])
if _lib is not None:
    _lib.ot_assoc_solve_eps_scaling.restype, _lib.ot_assoc_solve_eps_scaling.argtypes = \
        SIGNATURES["ot_assoc_solve_eps_scaling"]


def _ctx_solve_eps_scaling(self, C, p, q, eps, eps0, factor=0.3, tol_stage=1e-3, tol=1e-6, max_iter=2000,
                           warm_g=None, want_pi=False, want_load=True, stream=None):
    """Algorithm 1 at eps, started through the stages eps0 * factor^s (eps-scaling).
    Returns (Result, per-stage iteration counts)."""
    _need(C, torch.float32, "C", 2)
    _need(p, torch.float32, "p", 1)
    _need(q, torch.float32, "q", 1)
    I, J = C.shape
    g = warm_g.clone() if warm_g is not None else None
    r, f, g, pi, load = self._result(I, J, C.device, want_pi, want_load, None, g)
    its = (ctypes.c_int32 * 64)()
    ns = ctypes.c_int32(0)
    st = self._L.ot_assoc_solve_eps_scaling(self._h, _ptr(C), C.stride(0), _ptr(p), _ptr(q), I, J, float(eps),
                                            float(eps0), float(factor), float(tol_stage), float(tol),
                                            int(max_iter), int(warm_g is not None), ctypes.byref(r), its,
                                            ctypes.byref(ns), _stream(stream))
    self._check(st, allow_nc=True)
    return self._pack(r, f, g, pi, load), list(its[:ns.value])


Context.solve_eps_scaling = _ctx_solve_eps_scaling


# ---- asynchronous solves -----------------------------------------------------------------------
SIGNATURES["ot_assoc_solve_cost_async"] = (ctypes.c_int, [_VP, _VP, _I64, _VP, _VP, _I64, _I64, _D, _D, _I32, _I32,
                                                          ctypes.POINTER(ot_assoc_result),
                                                          ctypes.POINTER(ctypes.c_uint64), _VP])
SIGNATURES["ot_assoc_wait"] = (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.POINTER(ot_assoc_result)])
if _lib is not None:
    for _name in ("ot_assoc_solve_cost_async", "ot_assoc_wait"):
        _fn = getattr(_lib, _name)
        _fn.restype, _fn.argtypes = SIGNATURES[_name]


class Pending:
    """An enqueued solve (ot_assoc_solve_cost_async); wait() returns its Result."""

    def __init__(self, ctx, ticket, r, f, g, pi, load):
        self._ctx, self.ticket, self._r = ctx, ticket, r
        self._bufs = (f, g, pi, load)

    def wait(self) -> Result:
        st = self._ctx._L.ot_assoc_wait(self._ctx._h, self.ticket, ctypes.byref(self._r))
        self._ctx._check(st, allow_nc=True)
        return self._ctx._pack(self._r, *self._bufs)


def _ctx_solve_cost_async(self, C, p, q, eps, tol=1e-6, max_iter=2000, warm_g=None, want_pi=False, want_load=True,
                          f=None, g=None, stream=None) -> Pending:
    _need(C, torch.float32, "C", 2)
    _need(p, torch.float32, "p", 1)
    _need(q, torch.float32, "q", 1)
    I, J = C.shape
    if warm_g is not None:
        g = warm_g if g is None else g.copy_(warm_g)
    r, f, g, pi, load = self._result(I, J, C.device, want_pi, want_load, f, g)
    ticket = ctypes.c_uint64(0)
    st = self._L.ot_assoc_solve_cost_async(self._h, _ptr(C), C.stride(0), _ptr(p), _ptr(q), I, J, float(eps),
                                           float(tol), int(max_iter), int(warm_g is not None), ctypes.byref(r),
                                           ctypes.byref(ticket), _stream(stream))
    self._check(st)
    return Pending(self, ticket.value, r, f, g, pi, load)


Context.solve_cost_async = _ctx_solve_cost_async


# ---- several solves on one cost matrix ----------------------------------------------------------
SIGNATURES["ot_assoc_solve_cost_multi"] = (ctypes.c_int, [_VP, _VP, _I64, _VP, _VP, _I64, _I64, _I32, _PD, _PD, _I32,
                                                          ctypes.POINTER(ot_assoc_result), _VP])
if _lib is not None:
    _lib.ot_assoc_solve_cost_multi.restype, _lib.ot_assoc_solve_cost_multi.argtypes = \
        SIGNATURES["ot_assoc_solve_cost_multi"]


def _ctx_solve_cost_multi(self, C, p, q, eps, tol=1e-6, max_iter=2000, want_pi=False, want_load=True, fs=None,
                          gs=None, stream=None) -> list:
    """Up to three solves of Algorithm 1 on one C (eps sweep) in one launch; a Result each."""
    _need(C, torch.float32, "C", 2)
    _need(p, torch.float32, "p", 1)
    _need(q, torch.float32, "q", 1)
    I, J = C.shape
    eps = [float(e) for e in eps]
    n = len(eps)
    tols = [float(t) for t in (tol if isinstance(tol, (list, tuple)) else [tol] * n)]
    arr = (ot_assoc_result * max(n, 1))()
    keep = []
    for k in range(n):
        r, f, g, pi, load = self._result(I, J, C.device, want_pi, want_load, fs[k] if fs else None,
                                         gs[k] if gs else None)
        arr[k] = r
        keep.append((f, g, pi, load))
    e_arr = (ctypes.c_double * max(n, 1))(*eps)
    t_arr = (ctypes.c_double * max(n, 1))(*tols)
    st = self._L.ot_assoc_solve_cost_multi(self._h, _ptr(C), C.stride(0), _ptr(p), _ptr(q), I, J, n, e_arr, t_arr,
                                           int(max_iter), arr, _stream(stream))
    self._check(st, allow_nc=True)
    return [self._pack(arr[k], *keep[k]) for k in range(n)]


Context.solve_cost_multi = _ctx_solve_cost_multi


# ---- Euclidean cost formed inside the sweeps -------------------------------------------------------
SIGNATURES["ot_assoc_solve_euclid"] = (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _I64, _I64, _D, _D, _I32, _I32,
                                                      ctypes.POINTER(ot_assoc_result), _VP])
if _lib is not None:
    _lib.ot_assoc_solve_euclid.restype, _lib.ot_assoc_solve_euclid.argtypes = SIGNATURES["ot_assoc_solve_euclid"]


def _ctx_solve_euclid(self, dev_xy, rrh_xy, p, q, eps, tol=1e-6, max_iter=2000, warm_g=None, want_pi=False,
                      want_load=True, stream=None) -> Result:
    """Algorithm 1 with C_ij = ||x_i - x_j|| formed on the fly (no cost matrix)."""
    _need(dev_xy, torch.float32, "dev_xy", 2)
    _need(rrh_xy, torch.float32, "rrh_xy", 2)
    _need(p, torch.float32, "p", 1)
    _need(q, torch.float32, "q", 1)
    if not dev_xy.is_contiguous() or not rrh_xy.is_contiguous() or dev_xy.shape[1] != 2 or rrh_xy.shape[1] != 2:
        raise ValueError("coordinates must be contiguous (n, 2) tensors")
    I, J = dev_xy.shape[0], rrh_xy.shape[0]
    g = warm_g.clone() if warm_g is not None else None
    r, f, g, pi, load = self._result(I, J, dev_xy.device, want_pi, want_load, None, g)
    st = self._L.ot_assoc_solve_euclid(self._h, _ptr(dev_xy), _ptr(rrh_xy), _ptr(p), _ptr(q), I, J, float(eps),
                                       float(tol), int(max_iter), int(warm_g is not None), ctypes.byref(r),
                                       _stream(stream))
    self._check(st, allow_nc=True)
    return self._pack(r, f, g, pi, load)


Context.solve_euclid = _ctx_solve_euclid


# ---- rates and cost in one pass --------------------------------------------------------------------
SIGNATURES["ot_assoc_build_cost_from_gains"] = (ctypes.c_int, [_VP, _VP, _I64, _VP, _I64, _I64, _D, _D, _D, _VP,
                                                               _I64, _VP, _I64, _D, _PD, _VP])
if _lib is not None:
    _lib.ot_assoc_build_cost_from_gains.restype, _lib.ot_assoc_build_cost_from_gains.argtypes = \
        SIGNATURES["ot_assoc_build_cost_from_gains"]


def _ctx_build_cost_from_gains(self, G, P, N0, W_hz, mu, eps_rel=None, C_out=None, R_out=None, stream=None):
    """Rates (Sec. II-A) and cost 1/(mu R) in one pass over the gains; returns (C, eps or None)."""
    _need(G, torch.float32, "G", 2)
    _need(P, torch.float32, "P", 1)
    I, J = G.shape
    if C_out is None:
        C_out = torch.empty((I, J), dtype=torch.float32, device=G.device)
    _need(C_out, torch.float32, "C_out", 2)
    if R_out is not None:
        _need(R_out, torch.float32, "R_out", 2)
    eps = ctypes.c_double(0.0)
    self._check(self._L.ot_assoc_build_cost_from_gains(
        self._h, _ptr(G), G.stride(0), _ptr(P), I, J, float(N0), float(W_hz), float(mu), _ptr(R_out),
        R_out.stride(0) if R_out is not None else 0, _ptr(C_out), C_out.stride(0), float(eps_rel or 0.0),
        ctypes.byref(eps) if eps_rel is not None else None, _stream(stream)))
    return C_out, (eps.value if eps_rel is not None else None)


Context.build_cost_from_gains = _ctx_build_cost_from_gains


# ---- one time instance of a drifting cell -----------------------------------------------------------
SIGNATURES["ot_assoc_build_cost_mobile"] = (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _I64, _I64, _D, _D, _D,
                                                           _D, _D, _VP, _I64, _D, _PD, _VP])
if _lib is not None:
    _lib.ot_assoc_build_cost_mobile.restype, _lib.ot_assoc_build_cost_mobile.argtypes = \
        SIGNATURES["ot_assoc_build_cost_mobile"]


def _ctx_build_cost_mobile(self, dev_xy, dev_v, rrh_xy, shadow_db, P, dt, side_m, N0, W_hz, mu, C_out=None,
                           eps_rel=None, stream=None):
    """Move the devices by dt (dev_xy, dev_v updated in place) and rebuild C (rates of Sec. II-A,
    cost of Sec. IV); returns (C, eps or None)."""
    _need(dev_xy, torch.float64, "dev_xy", 2)
    _need(dev_v, torch.float64, "dev_v", 2)
    _need(rrh_xy, torch.float32, "rrh_xy", 2)
    _need(shadow_db, torch.float32, "shadow_db", 2)
    _need(P, torch.float32, "P", 1)
    I, J = shadow_db.shape
    if (dev_xy.shape != (I, 2) or dev_v.shape != (I, 2) or rrh_xy.shape != (J, 2) or P.shape[0] != J
            or not all(t.is_contiguous() for t in (dev_xy, dev_v, rrh_xy, shadow_db))):
        raise ValueError("dev_xy, dev_v (I, 2), rrh_xy (J, 2), shadow_db (I, J) contiguous, P (J,)")
    if C_out is None:
        C_out = torch.empty((I, J), dtype=torch.float32, device=shadow_db.device)
    _need(C_out, torch.float32, "C_out", 2)
    eps = ctypes.c_double(0.0)
    self._check(self._L.ot_assoc_build_cost_mobile(
        self._h, _ptr(dev_xy), _ptr(dev_v), _ptr(rrh_xy), _ptr(shadow_db), _ptr(P), I, J, float(dt), float(side_m),
        float(N0), float(W_hz), float(mu), _ptr(C_out), C_out.stride(0), float(eps_rel or 0.0),
        ctypes.byref(eps) if eps_rel is not None else None, _stream(stream)))
    return C_out, (eps.value if eps_rel is not None else None)


Context.build_cost_mobile = _ctx_build_cost_mobile


# ---- row-sharded Algorithm 1 (Sec. III-C): the steps of one iteration over a shard ----------
OT_SHARD_FIRST, OT_SHARD_ITER, OT_SHARD_COLMAX, OT_SHARD_COLSUM, OT_SHARD_FINAL = 0, 1, 2, 3, 4
_CI = ctypes.c_int
SIGNATURES["ot_assoc_shard_mass"] = (ctypes.c_int, [_VP, _VP, _I64, _VP, _I64, _VP, _VP])
SIGNATURES["ot_assoc_shard_sweep"] = (ctypes.c_int, [_VP, _CI, _VP, _I64, _VP, _I64, _I64, _D, _D, _VP, _VP, _VP,
                                                     _VP, _VP, _VP, _VP, _VP, _VP])
SIGNATURES["ot_assoc_shard_update"] = (ctypes.c_int, [_VP, _CI, _VP, _I64, _D, _VP, _VP, _VP, _VP, _VP, _VP, _I32,
                                                      _D, _I32, _VP, _VP])
SIGNATURES["ot_assoc_shard_finish"] = (ctypes.c_int, [_VP, _VP, _VP, _VP, _I64, _D, _D, _D, _VP, _VP, _VP, _VP,
                                                      _VP])
if _lib is not None:
    for _name in ("ot_assoc_shard_mass", "ot_assoc_shard_sweep", "ot_assoc_shard_update", "ot_assoc_shard_finish"):
        _fn = getattr(_lib, _name)
        _fn.restype, _fn.argtypes = SIGNATURES[_name]


def _ctx_shard_mass(self, p, q, out, stream=None) -> None:
    """out (3 doubles) = sum of p, sum of q, 1.0 when an entry is not positive and finite."""
    _need(p, torch.float32, "p", 1)
    _need(q, torch.float32, "q", 1)
    _need(out, torch.float64, "out", 1)
    self._check(self._L.ot_assoc_shard_mass(self._h, _ptr(p), p.numel(), _ptr(q), q.numel(), _ptr(out),
                                            _stream(stream)))


def _ctx_shard_sweep(self, mode, C, p, inv_mass, eps, G, F_in, F_out, colmax, col_out, row_out=None, f_out=None,
                     state=None, stream=None) -> None:
    """One sweep of Algorithm 1 over a shard's rows (mode OT_SHARD_*); F_in / F_out are float32
    (I, 2) row-potential pairs; every output is a caller tensor; with a loop state (float64, 4)
    the sweep does nothing once the loop has stopped."""
    _need(C, torch.float32, "C", 2)
    _need(p, torch.float32, "p", 1)
    _need(G, torch.float64, "G", 1)
    _need(col_out, torch.float64, "col_out", 1)
    for name, t in (("F_in", F_in), ("F_out", F_out)):
        if t is not None:
            _need(t, torch.float32, name, 2)
    I, J = C.shape
    self._check(self._L.ot_assoc_shard_sweep(
        self._h, int(mode), _ptr(C), C.stride(0), _ptr(p), I, J, float(inv_mass), float(eps), _ptr(G), _ptr(F_in),
        _ptr(F_out), _ptr(colmax), _ptr(col_out), _ptr(row_out), _ptr(f_out), _ptr(state), _stream(stream)))


def _ctx_shard_update(self, mode, q, inv_qmass, col, colmax, G_in, G_out, flag, err=None, it=0, tol_stop=0.0,
                      max_iter=0, state=None, stream=None) -> None:
    """Column update from the column sums of every shard; flag (int32, 1) is OR-ed on trouble.
    With a loop state (ITER): the loop test on the summed residual err first (see the header)."""
    _need(q, torch.float32, "q", 1)
    _need(flag, torch.int32, "flag", 1)
    self._check(self._L.ot_assoc_shard_update(self._h, int(mode), _ptr(q), q.numel(), float(inv_qmass), _ptr(col),
                                              _ptr(colmax), _ptr(G_in), _ptr(G_out), _ptr(flag), _ptr(err), int(it),
                                              float(tol_stop), int(max_iter), _ptr(state), _stream(stream)))


def _ctx_shard_finish(self, col2, row_err, q, mass, inv_qmass, eps, G, g_out, rho_out, summary, stream=None) -> None:
    """Totals of the finalize sweep: summary = (transport cost, row residual, column residual)."""
    _need(q, torch.float32, "q", 1)
    _need(summary, torch.float64, "summary", 1)
    self._check(self._L.ot_assoc_shard_finish(self._h, _ptr(col2), _ptr(row_err), _ptr(q), q.numel(), float(mass),
                                              float(inv_qmass), float(eps), _ptr(G), _ptr(g_out), _ptr(rho_out),
                                              _ptr(summary), _stream(stream)))


Context.shard_mass = _ctx_shard_mass
Context.shard_sweep = _ctx_shard_sweep
Context.shard_update = _ctx_shard_update
Context.shard_finish = _ctx_shard_finish


# ---- measurement: the SFU exp2 throughput ------------------------------------------------------
SIGNATURES["ot_assoc_measure_ex2_rate"] = (ctypes.c_int, [_VP, _PD, _VP])
if _lib is not None:
    _lib.ot_assoc_measure_ex2_rate.restype, _lib.ot_assoc_measure_ex2_rate.argtypes = \
        SIGNATURES["ot_assoc_measure_ex2_rate"]


def _ctx_measure_ex2_rate(self, stream=None) -> float:
    """FP32 exp2 results per second of the device (the per-cell exponential's ceiling)."""
    out = ctypes.c_double(0.0)
    self._check(self._L.ot_assoc_measure_ex2_rate(self._h, ctypes.byref(out), _stream(stream)))
    return out.value


Context.measure_ex2_rate = _ctx_measure_ex2_rate
