"""Thin ctypes binding of ``include/dtws.h`` (libdtws.so).

Argument marshalling only: every step of the search runs in the library's
CUDA kernels.  Functions keep the C names (``dtws_create``, ``dtws_query``,
...) and take plain pointers; :class:`Index` is a convenience wrapper that
accepts torch tensors (device or host) and NumPy arrays and uses torch only
for device memory and the current CUDA stream.

There is no CPU fallback: if the library is not built or cannot be loaded,
every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

DTWS_OK = 0
DTWS_EINVAL = 1
DTWS_ENOMEM = 2
DTWS_ECUDA = 3
DTWS_ENONFINITE = 4
DTWS_ETIMEOUT = 5
DTWS_ENOTIMPL = 6
DTWS_EOVERFLOW = 7
DTWS_M_MAX = 8192
DTWS_K_MAX = 64
DTWS_NOALLOC_M_MAX = 8192


class DtwsError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {strerror(status)} ({status})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


class dtws_options(ctypes.Structure):
    _fields_ = [
        ("delta", ctypes.c_float),
        ("alpha_per_m", ctypes.c_float),
        ("seed_random", ctypes.c_int32),
        ("seed_proposals", ctypes.c_int32),
        ("proxy_terms", ctypes.c_int32),
        ("ordering", ctypes.c_int32),
        ("timing", ctypes.c_int32),
        ("exact_envelope", ctypes.c_int32),
        ("batch_lanes", ctypes.c_int32),
        ("batch_graph", ctypes.c_int32),
        ("exclusion_zone", ctypes.c_int32),
        ("unnormalised", ctypes.c_int32),
        ("wait_limit_ns", ctypes.c_int64),
        ("rng_seed", ctypes.c_uint64),
    ]


class dtws_query_stats(ctypes.Structure):
    _fields_ = [
        ("windows", ctypes.c_int64),
        ("pass_kim", ctypes.c_int64),
        ("pass_keogh_q", ctypes.c_int64),
        ("pass_keogh_s", ctypes.c_int64),
        ("dtw_started", ctypes.c_int64),
        ("dtw_abandoned", ctypes.c_int64),
        ("dtw_cells", ctypes.c_int64),
        ("rescored", ctypes.c_int64),
        ("seed_bsf", ctypes.c_float),
        ("phase_ms", ctypes.c_float * 8),
        ("kernel_launches", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "phase_ms"}
        d["phase_ms"] = list(self.phase_ms)
        return d


PHASES = ["qprep", "seeds", "lb_scan", "order", "dtw", "finalize", "window_stats", "envelope"]

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_S = ctypes.c_int
_SIGS = {
    "dtws_default_options": (None, [_P]),
    "dtws_create": (_S, [_P, _I64, _P, _P]),
    "dtws_destroy": (_S, [_P]),
    "dtws_set_options": (_S, [_P, _P]),
    "dtws_get_options": (_S, [_P, _P]),
    "dtws_query": (_S, [_P, _P, _I32, _I32, _I32, _P, _P, _P]),
    "dtws_query_batch": (_S, [_P, _P, _P, _P, _P, _I32, _I32, _P, _P, _P]),
    "dtws_sync_status": (_S, [_P, _P]),
    "dtws_last_stats": (_S, [_P, _P]),
    "dtws_clear_cache": (_S, [_P]),
    "dtws_strerror": (ctypes.c_char_p, [_S]),
    "dtws_last_error_detail": (ctypes.c_char_p, []),
    "dtws_debug_fail_next_allocs": (None, [ctypes.c_int]),
    "dtws_debug_set_xz_capacity": (_S, [_P, _I32, _I32]),
    "dtws_debug_set_pool_capacity": (_S, [_P, _I64]),
    "dtws_window_stats": (_S, [_P, _I32, _P, _P, _P, _P]),
    "dtws_series_envelope": (_S, [_P, _I32, _P, _P, _P]),
    "dtws_dtw_at": (_S, [_P, _P, _I32, _I32, _P, _I64, _P, _P]),
    "dtws_dtw_at_f64": (_S, [_P, _P, _I32, _I32, _P, _I64, _P, _P]),
    "dtws_lower_bounds_at": (_S, [_P, _P, _I32, _I32, _P, _I64, _P, _P, _P, _P]),
    "dtws_dtw_at_noalloc": (_S, [_P, _I64, _P, _I32, _I32, _P, _I64, _P, _P]),
    "dtws_debug_wait_selftest": (_S, [_P, _I64, _P]),
    "dtws_debug_lock_selftest": (_S, [_P, _I64, _P]),
    "dtws_autotune": (_S, [_P, _P, _P, _I32, _I32, _P]),
    "dtws_tune_entry": (_S, [_P, _I32, _I32, _P, _P]),
    "dtws_set_encoder": (_S, [_P, _P, _I32, _P]),
    "dtws_learned_embeddings": (_S, [_P, _I32, _P, _I64, _P]),
    "dtws_enc_prep": (_S, [_P, _I64, _P, _I32, _I32, _P, _P]),
    "dtws_enc_forward": (_S, [_P, _P, _I32, _P, _P]),
    "dtws_enc_loss_grad": (_S, [_P, _P, _P, _P, _I32, _P, _P, _P]),
    "dtws_trainer_create": (_S, [_P, _I32, _I32, _P, _P]),
    "dtws_trainer_step": (_S, [_P, _P, _P, _I64, _P, _P, _I32, _P, _I32, _P, _P]),
    "dtws_trainer_params": (_S, [_P, _P, _P]),
    "dtws_trainer_destroy": (_S, [_P]),
}

DTWS_ORDER_PLAIN = 0
DTWS_ORDER_LEARNED = 1
DTWS_ENC_PARAMS = 38112
DTWS_ENC_DIM = 64
DTWS_ENC_U = 64


class dtws_adam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libdtws.so (optionally building it first).  Raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(
                f"libdtws.so not found at {path}: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def exported_symbols() -> list[str]:
    return sorted(_SIGS)


def strerror(status: int) -> str:
    try:
        return load().dtws_strerror(status).decode()
    except RuntimeError:
        return f"status {status}"


def _check(status: int, where: str):
    if status != DTWS_OK:
        detail = load().dtws_last_error_detail().decode(errors="replace")
        raise DtwsError(status, where, detail)


# ------------------------------------------------------------------ C names
def dtws_default_options() -> dtws_options:
    o = dtws_options()
    load().dtws_default_options(ctypes.byref(o))
    return o


def dtws_create(series_ptr: int, n: int, stream: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().dtws_create(series_ptr, n, stream, ctypes.byref(h)), "dtws_create")
    return h


def dtws_destroy(h) -> None:
    _check(load().dtws_destroy(h), "dtws_destroy")


def dtws_set_options(h, opt: dtws_options) -> None:
    _check(load().dtws_set_options(h, ctypes.byref(opt)), "dtws_set_options")


def dtws_get_options(h) -> dtws_options:
    o = dtws_options()
    _check(load().dtws_get_options(h, ctypes.byref(o)), "dtws_get_options")
    return o


def dtws_query(h, Q_ptr, m, r, k, idx_ptr, dist_ptr, stream=0) -> None:
    _check(load().dtws_query(h, Q_ptr, m, r, k, idx_ptr, dist_ptr, stream), "dtws_query")


def dtws_query_batch(h, Q_ptr, q_off_ptr, m_ptr, r_ptr, nq, k, idx_ptr, dist_ptr, stream=0) -> None:
    _check(load().dtws_query_batch(h, Q_ptr, q_off_ptr, m_ptr, r_ptr, nq, k, idx_ptr, dist_ptr, stream),
           "dtws_query_batch")


def dtws_sync_status(h, stream=0) -> int:
    return load().dtws_sync_status(h, stream)


def dtws_last_stats(h) -> dtws_query_stats:
    s = dtws_query_stats()
    _check(load().dtws_last_stats(h, ctypes.byref(s)), "dtws_last_stats")
    return s


def dtws_clear_cache(h) -> None:
    _check(load().dtws_clear_cache(h), "dtws_clear_cache")


def dtws_debug_fail_next_allocs(count: int) -> None:
    load().dtws_debug_fail_next_allocs(count)


# ------------------------------------------------------------------ wrapper
def _torch():
    import torch  # torch is plumbing here: device memory and streams
    return torch


_CUDA_AVAILABLE = None  # torch.cuda.is_available(), asked once per process


def _stream_ptr(stream) -> int:
    global _CUDA_AVAILABLE
    if stream is None:
        torch = _torch()
        if _CUDA_AVAILABLE is None:
            _CUDA_AVAILABLE = bool(torch.cuda.is_available())
        return int(torch.cuda.current_stream().cuda_stream) if _CUDA_AVAILABLE else 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def apply_options(o: dtws_options, kw: dict) -> dtws_options:
    """Set the named fields of a dtws_options; an unknown name raises
    (a ctypes structure would otherwise take it as a plain attribute and the
    library would never see it)."""
    fields = {f for f, _ in dtws_options._fields_}
    unknown = sorted(set(kw) - fields)
    if unknown:
        raise KeyError(f"unknown dtws_options field(s): {', '.join(unknown)}")
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class _Arg:
    """Pointer to an array's data: a contiguous torch tensor (any device) or
    a NumPy array kept alive for the call."""

    def __init__(self, a, dtype):
        torch = _torch()
        if isinstance(a, torch.Tensor):
            want = {np.float32: torch.float32, np.float64: torch.float64, np.int64: torch.int64,
                    np.int32: torch.int32}[dtype]
            if a.dtype != want:
                a = a.to(want)
            self.obj = a.contiguous()
            self.ptr = self.obj.data_ptr()
            self.size = self.obj.numel()
        else:
            self.obj = np.ascontiguousarray(a, dtype=dtype)
            self.ptr = self.obj.ctypes.data
            self.size = self.obj.size


class Index:
    """A search handle over one series (``dtws_create`` / ``dtws_destroy``)."""

    def __init__(self, series, stream=None, options: dict | None = None):
        self._lib = load()
        a = _Arg(series, np.float32)
        self.n = a.size
        self.h = dtws_create(a.ptr, a.size, _stream_ptr(stream))
        if options:
            self.set_options(**options)

    def close(self):
        if getattr(self, "h", None):
            dtws_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_options(self, **kw):
        o = dtws_get_options(self.h)
        apply_options(o, kw)
        dtws_set_options(self.h, o)

    def options(self) -> dict:
        o = dtws_get_options(self.h)
        return {f: getattr(o, f) for f, _ in o._fields_}

    # -------------------------------------------------------------- search
    def query(self, Q, r: int, k: int = 1, out=None, stream=None):
        """Top-k (offsets int64, squared DTW float32).  ``out`` = (idx, dist)
        tensors to write into (device or host); default: host NumPy arrays."""
        q = _Arg(Q, np.float32)
        if out is None:
            idx = np.empty(k, np.int64)
            dist = np.empty(k, np.float32)
            ip, dp = idx.ctypes.data, dist.ctypes.data
        else:
            idx, dist = out
            ip, dp = idx.data_ptr(), dist.data_ptr()
        dtws_query(self.h, q.ptr, q.size, r, k, ip, dp, _stream_ptr(stream))
        return idx, dist

    def query_batch(self, queries, rs, k: int = 1, stream=None):
        """Many queries; returns ([nq, k] offsets, [nq, k] distances), host."""
        ms = np.array([len(q) for q in queries], np.int32)
        off = np.zeros(len(queries) + 1, np.int64)
        off[1:] = np.cumsum(ms)
        cat = np.concatenate([np.asarray(q, np.float32) for q in queries]) \
            if not hasattr(queries, "data_ptr") else queries
        rr = np.ascontiguousarray(rs, dtype=np.int32)
        c = _Arg(cat, np.float32)
        nq = len(queries)
        idx = np.empty((nq, k), np.int64)
        dist = np.empty((nq, k), np.float32)
        dtws_query_batch(self.h, c.ptr, off.ctypes.data, ms.ctypes.data, rr.ctypes.data, nq, k,
                         idx.ctypes.data, dist.ctypes.data, _stream_ptr(stream))
        return idx, dist

    def sync_status(self, stream=None) -> int:
        return dtws_sync_status(self.h, _stream_ptr(stream))

    def last_stats(self) -> dict:
        return dtws_last_stats(self.h).as_dict()

    def clear_cache(self):
        dtws_clear_cache(self.h)

    # -------------------------------------------------------------- building blocks
    def window_stats(self, m: int, stream=None):
        N = self.n - m + 1
        mh, ml, inv = (np.empty(N, np.float32) for _ in range(3))
        _check(self._lib.dtws_window_stats(self.h, m, mh.ctypes.data, ml.ctypes.data, inv.ctypes.data,
                                           _stream_ptr(stream)), "dtws_window_stats")
        return mh, ml, inv

    def series_envelope(self, r: int, stream=None):
        U = np.empty(self.n, np.float32)
        L = np.empty(self.n, np.float32)
        _check(self._lib.dtws_series_envelope(self.h, r, U.ctypes.data, L.ctypes.data, _stream_ptr(stream)),
               "dtws_series_envelope")
        return U, L

    def dtw_at(self, Q, r: int, offsets, stream=None) -> np.ndarray:
        q = _Arg(Q, np.float32)
        o = _Arg(offsets, np.int64)
        out = np.empty(o.size, np.float32)
        _check(self._lib.dtws_dtw_at(self.h, q.ptr, q.size, r, o.ptr, o.size, out.ctypes.data,
                                     _stream_ptr(stream)), "dtws_dtw_at")
        return out

    def dtw_at_f64(self, Q, r: int, offsets, stream=None) -> np.ndarray:
        q = _Arg(Q, np.float32)
        o = _Arg(offsets, np.int64)
        out = np.empty(o.size, np.float64)
        _check(self._lib.dtws_dtw_at_f64(self.h, q.ptr, q.size, r, o.ptr, o.size, out.ctypes.data,
                                         _stream_ptr(stream)), "dtws_dtw_at_f64")
        return out

    def debug_set_pool_capacity(self, cap: int):
        """Test hook: survivor pool capacity of the batch's persistent stage
        (0: none, -1: default; see dtws.h)."""
        _check(self._lib.dtws_debug_set_pool_capacity(self.h, cap), "dtws_debug_set_pool_capacity")

    def debug_set_xz_capacity(self, buf_cap: int, sel_cap: int):
        """Test hook: capacities of the wide exclusion zone's candidate buffer
        and re-score list (see dtws.h)."""
        _check(self._lib.dtws_debug_set_xz_capacity(self.h, buf_cap, sel_cap), "dtws_debug_set_xz_capacity")

    def debug_lock_selftest(self, wait_ns: int, stream=None):
        _check(self._lib.dtws_debug_lock_selftest(self.h, wait_ns, _stream_ptr(stream)), "dtws_debug_lock_selftest")

    def debug_wait_selftest(self, wait_ns: int, stream=None):
        _check(self._lib.dtws_debug_wait_selftest(self.h, wait_ns, _stream_ptr(stream)), "dtws_debug_wait_selftest")

    def autotune(self, ms, rs, samples: int = 4096, stream=None):
        """Tune the survivor-DTW kernel shape for each (m, r) pair."""
        mm = np.ascontiguousarray(ms, dtype=np.int32)
        rr = np.ascontiguousarray(rs, dtype=np.int32)
        _check(self._lib.dtws_autotune(self.h, mm.ctypes.data, rr.ctypes.data, mm.size, samples,
                                       _stream_ptr(stream)), "dtws_autotune")

    def tune_entry(self, m: int, r: int):
        """(L, K, warps, ms_default, ms_best) of a tuned (m, r)."""
        shape = np.zeros(3, np.int32)
        ms = np.zeros(2, np.float32)
        _check(self._lib.dtws_tune_entry(self.h, m, r, shape.ctypes.data, ms.ctypes.data), "dtws_tune_entry")
        return int(shape[0]), int(shape[1]), int(shape[2]), float(ms[0]), float(ms[1])

    def set_encoder(self, params, stream=None):
        p = _Arg(params, np.float32)
        _check(self._lib.dtws_set_encoder(self.h, p.ptr, p.size, _stream_ptr(stream)), "dtws_set_encoder")

    def learned_embeddings(self, m: int, stream=None) -> np.ndarray:
        b = m // 64
        rows = (self.n - m) // b + 1
        out = np.empty((rows, DTWS_ENC_DIM), np.float32)
        _check(self._lib.dtws_learned_embeddings(self.h, m, out.ctypes.data, rows, _stream_ptr(stream)),
               "dtws_learned_embeddings")
        return out

    def lower_bounds_at(self, Q, r: int, offsets, stream=None):
        q = _Arg(Q, np.float32)
        o = _Arg(offsets, np.int64)
        kim, kq, ks = (np.empty(o.size, np.float32) for _ in range(3))
        _check(self._lib.dtws_lower_bounds_at(self.h, q.ptr, q.size, r, o.ptr, o.size, kim.ctypes.data,
                                              kq.ctypes.data, ks.ctypes.data, _stream_ptr(stream)),
               "dtws_lower_bounds_at")
        return kim, kq, ks


# ------------------------------------------------------------------ learned proposals
def enc_prep(X, offsets, m: int, stream=None) -> np.ndarray:
    """u [rows][64] of the windows X[offsets[i]:offsets[i]+m] (dtws_enc_prep)."""
    x = _Arg(X, np.float32)
    o = np.ascontiguousarray(offsets, dtype=np.int64)
    u = np.empty((o.size, DTWS_ENC_U), np.float32)
    _check(load().dtws_enc_prep(x.ptr, x.size, o.ctypes.data, o.size, m, u.ctypes.data, _stream_ptr(stream)),
           "dtws_enc_prep")
    return u


def enc_forward(params, u, stream=None) -> np.ndarray:
    """Embeddings [rows][64] of u [rows][64] (dtws_enc_forward)."""
    p = _Arg(params, np.float32)
    uu = _Arg(u, np.float32)
    rows = uu.size // DTWS_ENC_U
    e = np.empty((rows, DTWS_ENC_DIM), np.float32)
    _check(load().dtws_enc_forward(p.ptr, uu.ptr, rows, e.ctypes.data, _stream_ptr(stream)), "dtws_enc_forward")
    return e


def enc_loss_grad(params, uq, uc, y, stream=None):
    """(mean loss, gradient [38112]) of a batch of triples (dtws_enc_loss_grad)."""
    p = _Arg(params, np.float32)
    a, b = _Arg(uq, np.float32), _Arg(uc, np.float32)
    yy = _Arg(y, np.float32)
    loss = np.zeros(1, np.float32)
    grad = np.empty(DTWS_ENC_PARAMS, np.float32)
    _check(load().dtws_enc_loss_grad(p.ptr, a.ptr, b.ptr, yy.ptr, yy.size, loss.ctypes.data, grad.ctypes.data,
                                     _stream_ptr(stream)), "dtws_enc_loss_grad")
    return float(loss[0]), grad


class Trainer:
    """Adam on the GPU over the encoder parameters (dtws_trainer_*)."""

    def __init__(self, params, max_batch: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self._lib = load()
        p = _Arg(params, np.float32)
        hp = dtws_adam(lr, beta1, beta2, eps)
        self.h = ctypes.c_void_p()
        _check(self._lib.dtws_trainer_create(p.ptr, p.size, max_batch, ctypes.byref(hp), ctypes.byref(self.h)),
               "dtws_trainer_create")

    def step(self, xq, xc, q_off, c_off, m: int, y, want_loss=True, stream=None):
        """xq, xc: device tensors (series); q_off, c_off, y: host arrays."""
        a, b = _Arg(xq, np.float32), _Arg(xc, np.float32)
        qo = np.ascontiguousarray(q_off, dtype=np.int64)
        co = np.ascontiguousarray(c_off, dtype=np.int64)
        yy = np.ascontiguousarray(y, dtype=np.float32)
        loss = np.zeros(1, np.float32)
        _check(self._lib.dtws_trainer_step(self.h, a.ptr, b.ptr, a.size, qo.ctypes.data, co.ctypes.data, m,
                                           yy.ctypes.data, yy.size, loss.ctypes.data if want_loss else None,
                                           _stream_ptr(stream)), "dtws_trainer_step")
        return float(loss[0]) if want_loss else None

    def params(self, stream=None) -> np.ndarray:
        out = np.empty(DTWS_ENC_PARAMS, np.float32)
        _check(self._lib.dtws_trainer_params(self.h, out.ctypes.data, _stream_ptr(stream)), "dtws_trainer_params")
        return out

    def close(self):
        if getattr(self, "h", None):
            self._lib.dtws_trainer_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
