"""ctypes binding of libplc (include/plc.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
Field arguments are contiguous CUDA tensors of shape (n, n, n) in [z][y][x]
order; PyTorch supplies device memory and the stream.  There is no CPU
fallback: if libplc.so is missing or cannot be loaded, `load()` raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libplc.so")

PLC_FP64, PLC_MIXED = 0, 1
STATUS = {0: "PLC_OK", 1: "PLC_ERR_INVALID_ARG", 2: "PLC_ERR_CUDA", 3: "PLC_ERR_NOT_CONVERGED",
          4: "PLC_ERR_NONFINITE", 5: "PLC_ERR_CG_BREAKDOWN", 6: "PLC_ERR_OOM"}

# Every symbol include/plc.h declares.
EXPORTS = ["plc_create", "plc_destroy", "plc_set_prior", "plc_prior_apply", "plc_logpost_grad",
           "plc_hessvec", "plc_default_opts", "plc_newton_krylov_map", "plc_map_vjp",
           "plc_gauss_map", "plc_wiener_lsq", "plc_set_bias", "plc_bias_logpost_grad",
           "plc_bias_hessvec", "plc_bias_map", "plc_compare", "plc_smooth", "plc_log_stats",
           "plc_set_fft_schedule", "plc_autotune",
           "plc_batch_create", "plc_batch_map", "plc_batch_destroy",
           "plc_profile_enable", "plc_profile_read", "plc_hessvec_noalloc", "plc_last_error",
           "plc_status_string"]


class PlcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_newton", ctypes.c_int), ("max_cg", ctypes.c_int),
                ("precond", ctypes.c_int), ("g0_norm", ctypes.c_double),
                ("step_cap", ctypes.c_double), ("eta_max", ctypes.c_double),
                ("cg_chunk", ctypes.c_int), ("mixed_switch", ctypes.c_double),
                ("device_driven", ctypes.c_int), ("start", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int), ("cg_iters", ctypes.c_int),
                ("hv_count", ctypes.c_int), ("grad_evals", ctypes.c_int),
                ("grad_ffts", ctypes.c_int), ("grad_ffts_fp64", ctypes.c_int),
                ("grad_rel", ctypes.c_double), ("g0_norm", ctypes.c_double),
                ("neg_logpost", ctypes.c_double), ("ms", ctypes.c_double),
                ("kernels", ctypes.c_longlong)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_longlong),
                ("timed", ctypes.c_longlong), ("total_ms", ctypes.c_double)]


_LIB: Optional[ctypes.CDLL] = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libplc.so and declare its signatures (raises if it is missing)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise ImportError(f"libplc.so not built at {path}; run python -m paper_0911_1407_gb300.build")
    lib = ctypes.CDLL(path)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, None
    DP = ctypes.POINTER(ctypes.c_double)
    sig = {
        "plc_create": (I, [ctypes.POINTER(P), I, D, I, P]),
        "plc_destroy": (I, [P]),
        "plc_set_prior": (I, [P, DP, DP, I, D, D]),
        "plc_prior_apply": (I, [P, P, P]),
        "plc_logpost_grad": (I, [P, P, P, P, D, DP, P]),
        "plc_hessvec": (I, [P, P, P, D, P, P]),
        "plc_default_opts": (I, [ctypes.POINTER(Opts)]),
        "plc_newton_krylov_map": (I, [P, P, P, D, P, ctypes.POINTER(Opts), ctypes.POINTER(Stats)]),
        "plc_map_vjp": (I, [P, P, P, D, P, P, DP, ctypes.POINTER(Opts), ctypes.POINTER(Stats)]),
        "plc_wiener_lsq": (I, [P, P, P, D, P, ctypes.POINTER(Opts), ctypes.POINTER(Stats)]),
        "plc_gauss_map": (I, [P, P, P, D, P, ctypes.POINTER(Opts), ctypes.POINTER(Stats)]),
        "plc_set_bias": (I, [P, DP, DP, I, D]),
        "plc_bias_logpost_grad": (I, [P, P, P, P, D, DP, P]),
        "plc_bias_hessvec": (I, [P, P, P, P, D, P, P]),
        "plc_bias_map": (I, [P, P, P, D, P, ctypes.POINTER(Opts), ctypes.POINTER(Stats)]),
        "plc_compare": (I, [P, P, P, DP, DP]),
        "plc_smooth": (I, [P, P, P, D]),
        "plc_log_stats": (I, [P, P, D, D, I, ctypes.POINTER(ctypes.c_longlong),
                              ctypes.POINTER(ctypes.c_longlong), DP]),
        "plc_set_fft_schedule": (I, [P, I, I]),
        "plc_autotune": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I), DP]),
        "plc_batch_create": (I, [ctypes.POINTER(P), ctypes.POINTER(P), I]),
        "plc_batch_map": (I, [P, ctypes.POINTER(P), ctypes.POINTER(P), DP, ctypes.POINTER(P),
                              ctypes.POINTER(Opts), ctypes.POINTER(Stats), P]),
        "plc_batch_destroy": (I, [P]),
        "plc_profile_enable": (I, [P, I]),
        "plc_profile_read": (I, [P, ctypes.POINTER(KernelTime), I, ctypes.POINTER(I)]),
        "plc_hessvec_noalloc": (I, [I, D, DP, DP, I, D, P, P, D, P, P, P]),
        "plc_last_error": (ctypes.c_char_p, [P]),
        "plc_status_string": (ctypes.c_char_p, [I]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    _LIB = lib
    return lib


def default_opts(**kw) -> Opts:
    o = Opts()
    load().plc_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _ptr(t: Optional[torch.Tensor], n: int, dtype, name: str, required: bool = True):
    if t is None:
        if required:
            raise ValueError(f"{name} is required")
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != (n, n, n) or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous ({n}, {n}, {n}) tensor")
    return ctypes.c_void_p(t.data_ptr())


def hessvec_noalloc(n: int, box: float, k, P, inv_lambda_dc: float, s: torch.Tensor,
                    w: Optional[torch.Tensor], nbar: float, v: torch.Tensor, out: torch.Tensor,
                    stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    """plc_hessvec_noalloc: FP64 H v for n <= 64 using the library's static
    scratch (for callers that cannot allocate device memory).  `out` must be
    supplied by the caller."""
    lib = load()
    k = np.ascontiguousarray(k, dtype=np.float64)
    P = np.ascontiguousarray(P, dtype=np.float64)
    DP = ctypes.POINTER(ctypes.c_double)
    stream = stream if stream is not None else torch.cuda.current_stream()
    st = lib.plc_hessvec_noalloc(int(n), float(box), k.ctypes.data_as(DP), P.ctypes.data_as(DP),
                                 int(k.size), float(inv_lambda_dc),
                                 _ptr(s, n, torch.float64, "s"), _ptr(w, n, torch.float64, "w", False),
                                 float(nbar), _ptr(v, n, torch.float64, "v"),
                                 _ptr(out, n, torch.float64, "out"),
                                 ctypes.c_void_p(stream.cuda_stream))
    if st != 0:
        raise PlcError(st, lib.plc_last_error(None).decode())
    return out


@dataclass
class MapResult:
    s: torch.Tensor
    status: int
    stats: dict


class Context:
    """One libplc context: a grid, a precision, a prior, on one CUDA stream."""

    def __init__(self, n: int, box: float, precision: str = "fp64",
                 stream: Optional[torch.cuda.Stream] = None):
        self.lib = load()
        self.n, self.box = int(n), float(box)
        self.precision = {"fp64": PLC_FP64, "mixed": PLC_MIXED}[precision]
        self.real = torch.float64 if self.precision == PLC_FP64 else torch.float32
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._h = ctypes.c_void_p()
        st = self.lib.plc_create(ctypes.byref(self._h), self.n, self.box, self.precision,
                                 ctypes.c_void_p(self.stream.cuda_stream))
        if st != 0:
            raise PlcError(st, self.lib.plc_last_error(None).decode())
        self.mu = None

    # -- plumbing ----------------------------------------------------------
    def _check(self, st: int, allow=(0,)) -> int:
        if st not in allow:
            raise PlcError(st, self.lib.plc_last_error(self._h).decode())
        return st

    def close(self):
        if self._h:
            self.lib.plc_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def field(self, dtype=None) -> torch.Tensor:
        return torch.empty((self.n,) * 3, dtype=dtype or self.real, device="cuda")

    # -- calls ---------------------------------------------------------------
    def set_prior(self, k, P, mu: float, inv_lambda_dc: float = 0.0):
        k = np.ascontiguousarray(k, dtype=np.float64)
        P = np.ascontiguousarray(P, dtype=np.float64)
        DP = ctypes.POINTER(ctypes.c_double)
        self._check(self.lib.plc_set_prior(self._h, k.ctypes.data_as(DP), P.ctypes.data_as(DP),
                                           int(k.size), float(mu), float(inv_lambda_dc)))
        self.mu = float(mu)
        self._prior = (k.copy(), P.copy(), float(mu), float(inv_lambda_dc))

    def prior_is(self, k, P, mu: float, inv_lambda_dc: float = 0.0) -> bool:
        """True when the last plc_set_prior on this context had these arguments."""
        cur = getattr(self, "_prior", None)
        return (cur is not None and cur[2] == float(mu) and cur[3] == float(inv_lambda_dc)
                and np.array_equal(cur[0], np.asarray(k, dtype=np.float64))
                and np.array_equal(cur[1], np.asarray(P, dtype=np.float64)))

    def prior_apply(self, x: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        out = self.field() if out is None else out
        self._check(self.lib.plc_prior_apply(self._h, _ptr(x, self.n, self.real, "x"),
                                             _ptr(out, self.n, self.real, "out")))
        return out

    def logpost_grad(self, s, N, w, nbar: float, grad: Optional[torch.Tensor] = None,
                     want_grad: bool = True):
        if want_grad and grad is None:
            grad = self.field()
        f = ctypes.c_double()
        self._check(self.lib.plc_logpost_grad(
            self._h, _ptr(s, self.n, self.real, "s"), _ptr(N, self.n, torch.int32, "N"),
            _ptr(w, self.n, self.real, "w", False), float(nbar), ctypes.byref(f),
            _ptr(grad, self.n, self.real, "grad", False)))
        return f.value, grad

    def hessvec(self, s, w, nbar: float, v, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        out = self.field() if out is None else out
        self._check(self.lib.plc_hessvec(
            self._h, _ptr(s, self.n, self.real, "s"), _ptr(w, self.n, self.real, "w", False),
            float(nbar), _ptr(v, self.n, self.real, "v"), _ptr(out, self.n, self.real, "Hv")))
        return out

    def newton_krylov_map(self, N, w, nbar: float, s: Optional[torch.Tensor] = None,
                          raise_on_fail: bool = True, **opts) -> MapResult:
        """MAP; s (float64) is the start point and is overwritten (default mu).
        With start=2, or with s omitted and start 1 (the default) or 2, the
        start is mu without an array holding it: s is output only."""
        if s is None:
            if self.mu is None:
                raise RuntimeError("set_prior first")
            if opts.get("start", 1) >= 1:
                s = torch.empty((self.n,) * 3, dtype=torch.float64, device="cuda")
                opts["start"] = 2
            else:
                s = torch.full((self.n,) * 3, self.mu, dtype=torch.float64, device="cuda")
        o, stt = default_opts(**opts), Stats()
        st = self.lib.plc_newton_krylov_map(
            self._h, _ptr(N, self.n, torch.int32, "N"), _ptr(w, self.n, torch.float64, "w", False),
            float(nbar), _ptr(s, self.n, torch.float64, "s"), ctypes.byref(o), ctypes.byref(stt))
        if raise_on_fail:
            self._check(st)
        return MapResult(s, st, stt.as_dict())

    def gauss_map(self, N, w, nbar: float, delta: Optional[torch.Tensor] = None,
                  raise_on_fail: bool = True, **opts) -> MapResult:
        """MAP of the Gaussian-prior Poisson model; delta (float64) is the
        start point (default 0) and is overwritten.  With start=2, or with
        delta omitted and start 1 (the default) or 2, the start is 0 without
        an array holding it: delta is output only."""
        if delta is None:
            if opts.get("start", 1) >= 1:
                delta = torch.empty((self.n,) * 3, dtype=torch.float64, device="cuda")
                opts["start"] = 2
            else:
                delta = torch.zeros((self.n,) * 3, dtype=torch.float64, device="cuda")
        o, stt = default_opts(**opts), Stats()
        st = self.lib.plc_gauss_map(
            self._h, _ptr(N, self.n, torch.int32, "N"), _ptr(w, self.n, torch.float64, "w", False),
            float(nbar), _ptr(delta, self.n, torch.float64, "delta"), ctypes.byref(o),
            ctypes.byref(stt))
        if raise_on_fail:
            self._check(st)
        return MapResult(delta, st, stt.as_dict())

    def wiener_lsq(self, N, w, nbar: float, out: Optional[torch.Tensor] = None,
                   raise_on_fail: bool = True, **opts):
        """LSQ-Wiener estimate of delta (float64 field); returns (delta, status, stats)."""
        out = self.field(torch.float64) if out is None else out
        o, stt = default_opts(**opts), Stats()
        st = self.lib.plc_wiener_lsq(
            self._h, _ptr(N, self.n, torch.int32, "N"), _ptr(w, self.n, torch.float64, "w", False),
            float(nbar), _ptr(out, self.n, torch.float64, "delta_out"), ctypes.byref(o),
            ctypes.byref(stt))
        if raise_on_fail:
            self._check(st)
        return out, st, stt.as_dict()

    # -- linear bias (Sec. 2.4.1) -------------------------------------------
    def set_bias(self, k, b, b_dc: float = 1.0):
        """Bias table b(k) (linear in ln k, ln b) and the DC multiplier."""
        k = np.ascontiguousarray(k, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        DP = ctypes.POINTER(ctypes.c_double)
        self._check(self.lib.plc_set_bias(self._h, k.ctypes.data_as(DP), b.ctypes.data_as(DP),
                                          int(k.size), float(b_dc)))

    def bias_logpost_grad(self, s, N, w, nbar: float, grad: Optional[torch.Tensor] = None,
                          want_grad: bool = True):
        """-ln P and its gradient with linear bias; s, grad in the context's
        precision, w float64 (or None)."""
        if want_grad and grad is None:
            grad = self.field()
        f = ctypes.c_double()
        self._check(self.lib.plc_bias_logpost_grad(
            self._h, _ptr(s, self.n, self.real, "s"), _ptr(N, self.n, torch.int32, "N"),
            _ptr(w, self.n, torch.float64, "w", False), float(nbar), ctypes.byref(f),
            _ptr(grad, self.n, self.real, "grad", False)))
        return f.value, grad

    def bias_hessvec(self, s, N, w, nbar: float, v, out: Optional[torch.Tensor] = None):
        """Exact Hessian of the linear-bias -ln P at s applied to v."""
        out = self.field() if out is None else out
        self._check(self.lib.plc_bias_hessvec(
            self._h, _ptr(s, self.n, self.real, "s"), _ptr(N, self.n, torch.int32, "N"),
            _ptr(w, self.n, torch.float64, "w", False), float(nbar),
            _ptr(v, self.n, self.real, "v"), _ptr(out, self.n, self.real, "Hv")))
        return out

    def bias_map(self, N, w, nbar: float, s: Optional[torch.Tensor] = None,
                 raise_on_fail: bool = True, **opts) -> MapResult:
        """MAP with linear bias; s (float64) is the start point (default 0,
        delta_M = 0) and is overwritten."""
        if s is None:
            s = torch.zeros((self.n,) * 3, dtype=torch.float64, device="cuda")
        o, stt = default_opts(**opts), Stats()
        st = self.lib.plc_bias_map(
            self._h, _ptr(N, self.n, torch.int32, "N"), _ptr(w, self.n, torch.float64, "w", False),
            float(nbar), _ptr(s, self.n, torch.float64, "s"), ctypes.byref(o), ctypes.byref(stt))
        if raise_on_fail:
            self._check(st)
        return MapResult(s, st, stt.as_dict())

    def compare(self, a, b):
        """(r, D_Euc) of two float64 fields."""
        r, d = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.plc_compare(self._h, _ptr(a, self.n, torch.float64, "a"),
                                         _ptr(b, self.n, torch.float64, "b"), ctypes.byref(r),
                                         ctypes.byref(d)))
        return r.value, d.value

    def smooth(self, x, radius: float, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Gaussian smoothing of a float64 field (radius in Mpc/h)."""
        out = self.field(torch.float64) if out is None else out
        self._check(self.lib.plc_smooth(self._h, _ptr(x, self.n, torch.float64, "x"),
                                        _ptr(out, self.n, torch.float64, "y"), float(radius)))
        return out

    def log_stats(self, delta, lo: float, width: float, nbins: int):
        """Histogram of ln(1 + delta), (below, above, invalid), moments."""
        counts = (ctypes.c_longlong * int(nbins))()
        outside = (ctypes.c_longlong * 3)()
        mom = (ctypes.c_double * 4)()
        self._check(self.lib.plc_log_stats(self._h, _ptr(delta, self.n, torch.float64, "delta"),
                                           float(lo), float(width), int(nbins), counts, outside,
                                           mom))
        return np.array(counts[:], dtype=np.int64), tuple(outside[:]), tuple(mom[:])

    def set_fft_schedule(self, f1: int, f2: int):
        """FP32 line-transform schedule: four-step n = f1 f2, or (0, 0) Stockham."""
        self._check(self.lib.plc_set_fft_schedule(self._h, int(f1), int(f2)))

    def autotune(self, reps: int = 20):
        """Time every FP32 schedule offered for n, keep the fastest; returns
        (f1, f2, microseconds per Hv)."""
        f1, f2, us = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        self._check(self.lib.plc_autotune(self._h, int(reps), ctypes.byref(f1), ctypes.byref(f2),
                                          ctypes.byref(us)))
        return f1.value, f2.value, us.value

    def profile_enable(self, timing: bool = True):
        """Reset the per-kernel counters; timing=True also times every launch."""
        self._check(self.lib.plc_profile_enable(self._h, int(bool(timing))))

    def profile_read(self) -> dict:
        """{kernel kind: (launches, timed launches, total ms)} since the last reset."""
        cnt = ctypes.c_int()
        self._check(self.lib.plc_profile_read(self._h, None, 0, ctypes.byref(cnt)))
        arr = (KernelTime * cnt.value)()
        self._check(self.lib.plc_profile_read(self._h, arr, cnt.value, ctypes.byref(cnt)))
        return {r.name.decode(): (r.launches, r.timed, r.total_ms) for r in arr}

    def map_vjp(self, s_map, w, nbar: float, u, raise_on_fail: bool = True, **opts):
        vjp_N = self.field(torch.float64)
        vjp_lnA = ctypes.c_double()
        o, stt = default_opts(**opts), Stats()
        st = self.lib.plc_map_vjp(
            self._h, _ptr(s_map, self.n, torch.float64, "s_map"),
            _ptr(w, self.n, torch.float64, "w", False), float(nbar),
            _ptr(u, self.n, torch.float64, "u"), _ptr(vjp_N, self.n, torch.float64, "vjp_N"),
            ctypes.byref(vjp_lnA), ctypes.byref(o), ctypes.byref(stt))
        if raise_on_fail:
            self._check(st)
        return vjp_N, vjp_lnA.value, stt.as_dict()


class Batch:
    """plc_batch: independent MAP solves of several contexts as one graph launch."""

    def __init__(self, contexts):
        self.lib = load()
        self.contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c._h.value for c in self.contexts])
        self._h = ctypes.c_void_p()
        st = self.lib.plc_batch_create(ctypes.byref(self._h), arr, len(self.contexts))
        if st != 0:
            raise PlcError(st, self.lib.plc_last_error(None).decode())

    def close(self):
        if self._h:
            self.lib.plc_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def map(self, N, w, nbar, s, stream: Optional[torch.cuda.Stream] = None,
            raise_on_fail: bool = True, **opts):
        """Solve every context i from s[i] (float64, overwritten by its MAP)
        with counts N[i] (int32), selection w[i] (float64 or None), nbar[i]."""
        m = len(self.contexts)
        if not (len(N) == len(nbar) == len(s) == m) or (w is not None and len(w) != m):
            raise ValueError("one N, w, nbar, s per context")
        Np = (ctypes.c_void_p * m)(*[_ptr(N[i], c.n, torch.int32, "N").value
                                     for i, c in enumerate(self.contexts)])
        wp = None
        if w is not None:
            wp = (ctypes.c_void_p * m)(*[(_ptr(w[i], c.n, torch.float64, "w", False) or
                                          ctypes.c_void_p()).value
                                         for i, c in enumerate(self.contexts)])
        sp = (ctypes.c_void_p * m)(*[_ptr(s[i], c.n, torch.float64, "s").value
                                     for i, c in enumerate(self.contexts)])
        nb = (ctypes.c_double * m)(*[float(x) for x in nbar])
        o, stt = default_opts(**opts), (Stats * m)()
        stream = stream if stream is not None else torch.cuda.current_stream()
        st = self.lib.plc_batch_map(self._h, Np, wp, nb, sp, ctypes.byref(o), stt,
                                    ctypes.c_void_p(stream.cuda_stream))
        if raise_on_fail and st != 0:
            raise PlcError(st, self.lib.plc_last_error(None).decode())
        return st, [x.as_dict() for x in stt]
