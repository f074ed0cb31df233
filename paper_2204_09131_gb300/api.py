"""Thin ctypes binding of libisycos.so (C ABI in include/isycos.h).

Every function keeps the C name and only marshals arguments: NumPy arrays for host buffers,
torch CUDA tensors (or raw integers) for device buffers and streams.  The GPU work happens
in the library; there is no CPU fallback -- loading fails loudly when the library is absent.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libisycos.so")

OK = 0
E_INVAL = -1
E_NOMEM = -2
E_CUDA = -3
E_TIMEOUT = -4
E_TRUNC = -5
E_AGAIN = -6
E_NOTFOUND = -7
E_CANCELED = -8
PENDING = 1
MAX_M = 16384
MAX_K = 8

OPT_KERNEL = 1
OPT_INCREMENTAL = 2
OPT_SERVE_SLOTS = 3
OPT_SERVE_QUEUE = 4
OPT_LANES = 5
OPT_ESTIMATOR = 6
OPT_SPECULATION = 7
OPT_BU_DEVICE = 8
OPT_TIME_LIMIT_MS = 9


class IsycosError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("isycos status %d: %s" % (status, msg))
        self.status = status


class isycos_window(ctypes.Structure):
    _fields_ = [("xs", ctypes.c_int32), ("ys", ctypes.c_int32), ("start", ctypes.c_int64),
                ("m", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class isycos_mi_out(ctypes.Structure):
    _fields_ = [("mi", ctypes.c_double), ("h_w", ctypes.c_double), ("nmi", ctypes.c_double),
                ("s_psi", ctypes.c_int64), ("s_log", ctypes.c_int64)]


class isycos_params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("score_kind", ctypes.c_int32), ("sigma", ctypes.c_double),
                ("tau", ctypes.c_double), ("s_min", ctypes.c_int32), ("s_max", ctypes.c_int32),
                ("delta_td", ctypes.c_int32), ("delta_bu", ctypes.c_int32), ("h", ctypes.c_int32),
                ("t_max_idle", ctypes.c_int32), ("p", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("pruning", ctypes.c_int32), ("max_steps", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("sel_partitions", ctypes.c_int32),
                ("sel_samples", ctypes.c_int32), ("sel_alpha", ctypes.c_double),
                ("sel_rho", ctypes.c_double), ("chunks", ctypes.c_int32),
                ("estimator", ctypes.c_int32)]


class isycos_tuning(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("sorted_buckets", ctypes.c_uint32),
                ("window_size", ctypes.c_int32 * 15), ("n_windows", ctypes.c_int32),
                ("brute_ms", ctypes.c_double * 15), ("sorted_ms", ctypes.c_double * 15),
                ("sort_min", ctypes.c_int32), ("nt_switch", ctypes.c_int32),
                ("cross_size", ctypes.c_int32 * 3), ("pad", ctypes.c_int32),
                ("cross_brute_ms", ctypes.c_double * 3), ("cross_sorted_ms", ctypes.c_double * 3),
                ("nt_ms", ctypes.c_double * 2)]


class isycos_query(ctypes.Structure):
    _fields_ = [("xs", ctypes.c_int32), ("ys", ctypes.c_int32), ("t_begin", ctypes.c_int64),
                ("t_end", ctypes.c_int64), ("params", isycos_params)]


class isycos_result_window(ctypes.Structure):
    _fields_ = [("t_s", ctypes.c_int64), ("t_e", ctypes.c_int64), ("score", ctypes.c_double),
                ("mi", ctypes.c_double)]


class isycos_stats(ctypes.Structure):
    _fields_ = [("windows", ctypes.c_int64), ("pairs", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("incr_windows", ctypes.c_int64), ("incr_full_points", ctypes.c_int64),
                ("queries_done", ctypes.c_int64), ("decided_windows", ctypes.c_int64),
                ("mi_kernel_ms", ctypes.c_double), ("mi_kernel_launches", ctypes.c_int64),
                ("windows_by_size", ctypes.c_int64 * 15), ("launches_by_size", ctypes.c_int64 * 15),
                ("launch_ms_by_size", ctypes.c_double * 15),
                ("decided_by_size", ctypes.c_int64 * 15), ("dev_queries", ctypes.c_int64),
                ("dev_rounds", ctypes.c_int64), ("dev_cycles", ctypes.c_int64 * 3),
                ("work_bf", ctypes.c_int64), ("work_scan", ctypes.c_int64),
                ("work_search", ctypes.c_int64), ("work_sort", ctypes.c_int64)]


# NumPy views of the C structs (same layout).
WINDOW_DTYPE = np.dtype([("xs", np.int32), ("ys", np.int32), ("start", np.int64),
                         ("m", np.int32), ("reserved", np.int32)])
MI_OUT_DTYPE = np.dtype([("mi", np.float64), ("h_w", np.float64), ("nmi", np.float64),
                         ("s_psi", np.int64), ("s_log", np.int64)])
RESULT_DTYPE = np.dtype([("t_s", np.int64), ("t_e", np.int64), ("score", np.float64),
                         ("mi", np.float64)])
assert WINDOW_DTYPE.itemsize == ctypes.sizeof(isycos_window) == 24
assert MI_OUT_DTYPE.itemsize == ctypes.sizeof(isycos_mi_out) == 40
assert RESULT_DTYPE.itemsize == ctypes.sizeof(isycos_result_window) == 32

# Every entry point of include/isycos.h with its ctypes signature.
_VP = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
SIGNATURES = {
    "isycos_create": (_I32, [ctypes.POINTER(_VP), _I32, _U64]),
    "isycos_destroy": (_I32, [_VP]),
    "isycos_last_error": (ctypes.c_char_p, [_VP]),
    "isycos_params_default": (None, [ctypes.POINTER(isycos_params)]),
    "isycos_put_series": (_I32, [_VP, _VP, _I64, _I32, ctypes.POINTER(_I32)]),
    "isycos_put_series_many": (_I32, [_VP, _I32, _VP, _VP, _I32, _VP]),
    "isycos_drop_series": (_I32, [_VP, _I32]),
    "isycos_series_info": (_I32, [_VP, _I32, ctypes.POINTER(_VP), ctypes.POINTER(_I64)]),
    "isycos_mi_windows": (_I32, [_VP, _VP, _I64, _I32, _VP, _VP]),
    "isycos_mi_windows_device": (_I32, [_VP, _VP, _I64, _I32, _I32, _VP, _VP]),
    "isycos_device_status": (_I32, [_VP, _VP]),
    "isycos_mi_windows_points": (_I32, [_VP, _VP, _I64, _I32, _VP, _VP, _VP, _VP, _VP]),
    "isycos_mi_windows_plain": (_I32, [_VP, _VP, _I64, _I32, _VP, _VP]),
    "isycos_mi_chain": (_I32, [_VP, _I32, _I32, _VP, _VP, _I64, _I32, _VP, _VP]),
    "isycos_search": (_I32, [_VP, _I32, _I32, _I64, _I64, ctypes.POINTER(isycos_params), _VP,
                             _I64, ctypes.POINTER(_I64)]),
    "isycos_search_many": (_I32, [_VP, _I64, _VP, _VP, _VP, _VP, ctypes.POINTER(isycos_params),
                                  _VP, _I64, _VP]),
    "isycos_search_queries": (_I32, [_VP, _I64, _VP, _VP, _I64, _VP]),
    "isycos_serve_submit": (_I32, [_VP, _I32, _I32, _I64, _I64, ctypes.POINTER(isycos_params),
                                   ctypes.POINTER(_U64)]),
    "isycos_serve_poll": (_I32, [_VP, _U64, _VP, _I64, ctypes.POINTER(_I64),
                                 ctypes.POINTER(ctypes.c_double)]),
    "isycos_serve_poll_ex": (_I32, [_VP, _U64, _VP, _I64, ctypes.POINTER(_I64),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "isycos_serve_cancel": (_I32, [_VP, _U64]),
    "isycos_get_stats": (_I32, [_VP, ctypes.POINTER(isycos_stats)]),
    "isycos_reset_stats": (_I32, [_VP]),
    "isycos_tables": (_I32, [_VP, _I32, _VP, _VP]),
    "isycos_set_option": (_I32, [_VP, _I32, _I64]),
    "isycos_autotune": (_I32, [_VP, _I32, _VP]),
    "isycos_get_tuning": (_I32, [_VP, _I32, _VP, _VP, _VP]),
    "isycos_mi_windows_noalloc": (_I32, [_VP, _VP, _I64, _VP, _VP, _I64, _I32, _I32, _VP, _VP]),
}

_lib = None


def lib():
    """Load libisycos.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libisycos.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):          # torch tensor
        return a.data_ptr()
    return a.ctypes.data


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream                # torch.cuda.Stream


def _check(ctx, st):
    if st < 0:
        raise IsycosError(st, isycos_last_error(ctx))
    return st


# ---------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def isycos_create(device: int = 0, mem_budget_bytes: int = 0):
    h = ctypes.c_void_p()
    st = lib().isycos_create(ctypes.byref(h), device, mem_budget_bytes)
    if st != OK:
        raise IsycosError(st, "isycos_create failed")
    return h


def isycos_destroy(ctx):
    return _check(ctx, lib().isycos_destroy(ctx))


def isycos_last_error(ctx) -> str:
    r = lib().isycos_last_error(ctx)
    return r.decode() if r else ""


def isycos_params_default(**overrides) -> isycos_params:
    p = isycos_params()
    lib().isycos_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def isycos_put_series(ctx, data) -> int:
    """Make a series resident: a float32 NumPy array (host) or torch CUDA tensor (device)."""
    sid = ctypes.c_int32()
    if hasattr(data, "data_ptr"):
        assert data.dtype.__str__() == "torch.float32" and data.is_contiguous()
        on_dev = 1 if data.is_cuda else 0
        n = data.numel()
        p = data.data_ptr()
    else:
        data = np.ascontiguousarray(data, dtype=np.float32)
        on_dev, n, p = 0, data.shape[0], data.ctypes.data
    _check(ctx, lib().isycos_put_series(ctx, p, n, on_dev, ctypes.byref(sid)))
    return sid.value


def isycos_put_series_many(ctx, arrays) -> list:
    """Make several series resident in one call (one synchronisation): float32 NumPy arrays
    (host) or torch CUDA tensors (device), all of the same kind."""
    keep, ptrs, ns, kinds = [], [], [], set()
    for a in arrays:
        if hasattr(a, "data_ptr"):
            assert a.dtype.__str__() == "torch.float32" and a.is_contiguous()
            kinds.add(1 if a.is_cuda else 0)
            ptrs.append(a.data_ptr())
            ns.append(a.numel())
        else:
            a = np.ascontiguousarray(a, dtype=np.float32)
            kinds.add(0)
            ptrs.append(a.ctypes.data)
            ns.append(a.shape[0])
        keep.append(a)
    if not ptrs:
        return []
    assert len(kinds) == 1, "all series in host memory or all on the device"
    p = np.array(ptrs, dtype=np.uint64)
    n = np.array(ns, dtype=np.int64)
    ids = np.zeros(len(ptrs), dtype=np.int32)
    _check(ctx, lib().isycos_put_series_many(ctx, len(ptrs), p.ctypes.data, n.ctypes.data, kinds.pop(),
                                             ids.ctypes.data))
    return [int(v) for v in ids]


def isycos_drop_series(ctx, sid: int):
    return _check(ctx, lib().isycos_drop_series(ctx, sid))


def isycos_series_info(ctx, sid: int):
    p = ctypes.c_void_p()
    n = ctypes.c_int64()
    _check(ctx, lib().isycos_series_info(ctx, sid, ctypes.byref(p), ctypes.byref(n)))
    return p.value, n.value


def windows_array(xs, ys, starts, sizes) -> np.ndarray:
    """Build a window list (structured array with the isycos_window layout)."""
    starts = np.asarray(starts, dtype=np.int64)
    w = np.zeros(starts.shape[0], dtype=WINDOW_DTYPE)
    w["xs"] = xs
    w["ys"] = ys
    w["start"] = starts
    w["m"] = sizes
    return w


def isycos_mi_windows(ctx, windows: np.ndarray, k: int, stream=None) -> np.ndarray:
    windows = np.ascontiguousarray(windows, dtype=WINDOW_DTYPE)
    out = np.empty(windows.shape[0], dtype=MI_OUT_DTYPE)
    _check(ctx, lib().isycos_mi_windows(ctx, _ptr(windows), windows.shape[0], k, _ptr(out),
                                        _stream(stream)))
    return out


def isycos_mi_windows_device(ctx, d_windows, n_w: int, k: int, max_m: int, d_out, stream=None):
    """Device arrays (torch tensors or raw addresses); asynchronous on `stream`."""
    return _check(ctx, lib().isycos_mi_windows_device(ctx, _ptr(d_windows), n_w, k, max_m,
                                                      _ptr(d_out), _stream(stream)))


def isycos_device_status(ctx, stream=None):
    return _check(ctx, lib().isycos_device_status(ctx, _stream(stream)))


def isycos_mi_windows_points(ctx, windows: np.ndarray, k: int, stream=None):
    windows = np.ascontiguousarray(windows, dtype=WINDOW_DTYPE)
    total = int(windows["m"].astype(np.int64).sum())
    out = np.empty(windows.shape[0], dtype=MI_OUT_DTYPE)
    nx = np.empty(total, dtype=np.int32)
    ny = np.empty(total, dtype=np.int32)
    c = np.empty(total, dtype=np.int32)
    _check(ctx, lib().isycos_mi_windows_points(ctx, _ptr(windows), windows.shape[0], k, _ptr(out),
                                               _ptr(nx), _ptr(ny), _ptr(c), _stream(stream)))
    return out, nx, ny, c


def isycos_mi_windows_plain(ctx, windows: np.ndarray, k: int, stream=None) -> np.ndarray:
    windows = np.ascontiguousarray(windows, dtype=WINDOW_DTYPE)
    out = np.empty(windows.shape[0], dtype=MI_OUT_DTYPE)
    _check(ctx, lib().isycos_mi_windows_plain(ctx, _ptr(windows), windows.shape[0], k, _ptr(out),
                                              _stream(stream)))
    return out


def isycos_mi_chain(ctx, xs: int, ys: int, starts, sizes, k: int, stream=None) -> np.ndarray:
    starts = np.ascontiguousarray(starts, dtype=np.int64)
    sizes = np.ascontiguousarray(sizes, dtype=np.int32)
    out = np.empty(starts.shape[0], dtype=MI_OUT_DTYPE)
    _check(ctx, lib().isycos_mi_chain(ctx, xs, ys, _ptr(starts), _ptr(sizes), starts.shape[0], k,
                                      _ptr(out), _stream(stream)))
    return out


def _as_params(params):
    if params is None:
        return isycos_params_default()
    if isinstance(params, dict):
        return isycos_params_default(**params)
    return params


def isycos_search(ctx, xs: int, ys: int, t_begin: int, t_end: int, params=None,
                  cap: int = 1 << 16) -> np.ndarray:
    p = _as_params(params)
    out = np.empty(cap, dtype=RESULT_DTYPE)
    n = ctypes.c_int64()
    _check(ctx, lib().isycos_search(ctx, xs, ys, t_begin, t_end, ctypes.byref(p), _ptr(out), cap,
                                    ctypes.byref(n)))
    return out[:n.value].copy()


def isycos_search_many(ctx, xs, ys, t_begin, t_end, params=None, cap_per_query: int = 4096):
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    tb = np.ascontiguousarray(t_begin, dtype=np.int64)
    te = np.ascontiguousarray(t_end, dtype=np.int64)
    nq = xs.shape[0]
    p = _as_params(params)
    out = np.empty(max(nq * cap_per_query, 1), dtype=RESULT_DTYPE)
    n_out = np.zeros(nq, dtype=np.int64)
    _check(ctx, lib().isycos_search_many(ctx, nq, _ptr(xs), _ptr(ys), _ptr(tb), _ptr(te),
                                         ctypes.byref(p), _ptr(out), cap_per_query, _ptr(n_out)))
    return [out[q * cap_per_query: q * cap_per_query + n_out[q]].copy() for q in range(nq)]


def isycos_search_queries(ctx, queries, cap_per_query: int = 4096):
    """queries: list of (xs, ys, t_begin, t_end, params)."""
    nq = len(queries)
    arr = (isycos_query * max(nq, 1))()
    for i, (a, b, lo, hi, prm) in enumerate(queries):
        arr[i].xs, arr[i].ys, arr[i].t_begin, arr[i].t_end = a, b, lo, hi
        arr[i].params = _as_params(prm)
    out = np.empty(max(nq * cap_per_query, 1), dtype=RESULT_DTYPE)
    n_out = np.zeros(max(nq, 1), dtype=np.int64)
    _check(ctx, lib().isycos_search_queries(ctx, nq, ctypes.addressof(arr), _ptr(out),
                                            cap_per_query, _ptr(n_out)))
    return [out[q * cap_per_query: q * cap_per_query + n_out[q]].copy() for q in range(nq)]


def isycos_serve_submit(ctx, xs: int, ys: int, t_begin: int, t_end: int, params=None) -> int:
    p = _as_params(params)
    t = ctypes.c_uint64()
    _check(ctx, lib().isycos_serve_submit(ctx, xs, ys, t_begin, t_end, ctypes.byref(p),
                                          ctypes.byref(t)))
    return t.value


def isycos_serve_poll_ex(ctx, ticket: int, cap: int = 1024):
    """Returns None while pending, else (windows, latency_ms, admission_wait_ms)."""
    while True:
        out = np.empty(cap, dtype=RESULT_DTYPE)
        n = ctypes.c_int64()
        lat = ctypes.c_double()
        wait = ctypes.c_double()
        st = lib().isycos_serve_poll_ex(ctx, ticket, _ptr(out), cap, ctypes.byref(n), ctypes.byref(lat),
                                        ctypes.byref(wait))
        if st == PENDING:
            return None
        if st == E_TRUNC and n.value > cap:
            cap = int(n.value)
            continue
        _check(ctx, st)
        return out[:n.value].copy(), lat.value, wait.value


def isycos_serve_poll(ctx, ticket: int, cap: int = 1024):
    """Returns None while pending, else (windows, latency_ms).  A result larger than `cap`
    is fetched again with the size the library reports."""
    while True:
        out = np.empty(cap, dtype=RESULT_DTYPE)
        n = ctypes.c_int64()
        lat = ctypes.c_double()
        st = lib().isycos_serve_poll(ctx, ticket, _ptr(out), cap, ctypes.byref(n), ctypes.byref(lat))
        if st == PENDING:
            return None
        if st == E_TRUNC and n.value > cap:
            cap = int(n.value)
            continue
        _check(ctx, st)
        return out[:n.value].copy(), lat.value


def isycos_serve_cancel(ctx, ticket: int):
    return _check(ctx, lib().isycos_serve_cancel(ctx, ticket))


def isycos_get_stats(ctx) -> dict:
    s = isycos_stats()
    _check(ctx, lib().isycos_get_stats(ctx, ctypes.byref(s)))
    out = {}
    for f, _ in isycos_stats._fields_:
        v = getattr(s, f)
        out[f] = list(v) if isinstance(v, ctypes.Array) else v
    return out


def isycos_reset_stats(ctx):
    return _check(ctx, lib().isycos_reset_stats(ctx))


def isycos_tables(ctx, n_max: int):
    psi = np.empty(n_max + 1, dtype=np.int64)
    lg = np.empty(n_max + 1, dtype=np.int64)
    _check(ctx, lib().isycos_tables(ctx, n_max, _ptr(psi), _ptr(lg)))
    return psi, lg


def isycos_set_option(ctx, option: int, value: int):
    return _check(ctx, lib().isycos_set_option(ctx, option, value))


def isycos_autotune(ctx, k: int = 4) -> dict:
    """Time the brute-force and sorted MI paths per eligible size bucket and keep the faster;
    returns the probe sizes, times and the chosen sorted buckets."""
    t = isycos_tuning()
    _check(ctx, lib().isycos_autotune(ctx, k, ctypes.byref(t)))
    buckets = [b for b in range(15) if t.window_size[b]]
    cross = [i for i in range(3) if t.cross_size[i]]
    return {"k": t.k, "n_windows": t.n_windows,
            "sorted_buckets": [b for b in range(15) if (t.sorted_buckets >> b) & 1],
            "window_size": {b: t.window_size[b] for b in buckets},
            "brute_ms": {b: round(t.brute_ms[b], 4) for b in buckets},
            "sorted_ms": {b: round(t.sorted_ms[b], 4) for b in buckets},
            "sort_min": t.sort_min, "nt_switch": t.nt_switch,
            "crossover": {t.cross_size[i]: {"brute_ms": round(t.cross_brute_ms[i], 4),
                                            "sorted_ms": round(t.cross_sorted_ms[i], 4)} for i in cross},
            "nt_ms": {"256": round(t.nt_ms[0], 4), "1024": round(t.nt_ms[1], 4)}}


def isycos_get_tuning(ctx, k: int = 4):
    """The tuning the context uses for k, or None when k is not tuned."""
    sb, smin, nts = ctypes.c_uint32(), ctypes.c_int32(), ctypes.c_int32()
    st = lib().isycos_get_tuning(ctx, k, ctypes.byref(sb), ctypes.byref(smin), ctypes.byref(nts))
    if st == E_NOTFOUND:
        return None
    _check(ctx, st)
    return {"sorted_buckets": [b for b in range(15) if (sb.value >> b) & 1], "sort_min": smin.value,
            "nt_switch": nts.value}


class Context:
    """Owns an isycos context; closes it on exit."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        self.h = isycos_create(device, mem_budget_bytes)

    def close(self):
        if self.h is not None:
            isycos_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self.h

    def __exit__(self, *exc):
        self.close()
        return False
