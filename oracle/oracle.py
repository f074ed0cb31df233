"""Python view of the CPU oracle (``isycos_oracle.c``) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference leg may import this module.  The product package never imports it.

The oracle follows arXiv 2204.09131: the KSG estimator of Sec. 4.2 (Eq. KSGmi) with the
counting rule of the Sec. 7.1 example, the normalised score of Sec. 5.4, SYCOS_TD
(Algorithm 1), SYCOS_BU (Algorithm 2) and the noise pruning of Sec. 6.  The C file's
header lists the arithmetic contract.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "isycos_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# gcc flags: no fast-math, no contraction, no flush-to-zero.
CFLAGS = ["-O2", "-fno-fast-math", "-ffp-contract=off", "-std=c11", "-shared", "-fPIC"]

MUTATIONS = {
    "none": 0,
    "drop_inv_k": 1,
    "strict_count": 2,
    "count_self": 3,
    "psi_plus_one": 4,
    "swap_ny": 5,
    "tie_late": 6,
    "euclid": 7,
    "h_sign": 8,
    "psi_m_minus": 9,
    "accept_ge": 10,
    "tie_last": 11,
    "td_no_clamp": 12,
    "td_delta_overlap": 13,
    "noise_no_io": 14,
    "bu_square": 15,
    "bu_drop_both": 16,
    "no_history": 17,
    "chunk_no_overlap": 18,
    "runtime_windows": 19,
    "tiny_test": 20,
    "run_no_reset": 21,
    "bu_run_no_reset": 22,
    "td_tail": 23,
    "sample_draw": 24,
}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` if it is missing or stale."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + ".tmp%d" % os.getpid()
            cmd = ["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


class OrcMI(ctypes.Structure):
    _fields_ = [
        ("mi", ctypes.c_double),
        ("h_w", ctypes.c_double),
        ("nmi", ctypes.c_double),
        ("s_psi", ctypes.c_int64),
        ("s_log", ctypes.c_int64),
        ("mi_exact", ctypes.c_double),
        ("h_exact", ctypes.c_double),
    ]


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_int32),
        ("score_kind", ctypes.c_int32),
        ("sigma", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("s_min", ctypes.c_int32),
        ("s_max", ctypes.c_int32),
        ("delta_td", ctypes.c_int32),
        ("delta_bu", ctypes.c_int32),
        ("h", ctypes.c_int32),
        ("t_max_idle", ctypes.c_int32),
        ("p", ctypes.c_int32),
        ("pruning", ctypes.c_int32),
        ("max_steps", ctypes.c_int32),
        ("chunks", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
    ]


class OrcWindow(ctypes.Structure):
    _fields_ = [
        ("t_s", ctypes.c_int64),
        ("t_e", ctypes.c_int64),
        ("score", ctypes.c_double),
        ("mi", ctypes.c_double),
    ]


class OrcSeriesScorer(ctypes.Structure):
    _fields_ = [
        ("x", ctypes.c_void_p),
        ("y", ctypes.c_void_p),
        ("n", ctypes.c_int64),
        ("k", ctypes.c_int32),
        ("score_kind", ctypes.c_int32),
        ("evals", ctypes.c_int64),
        ("estimator", ctypes.c_int32),
        ("pad", ctypes.c_int32),
    ]


class OrcSelectParams(ctypes.Structure):
    _fields_ = [("partitions", ctypes.c_int32), ("samples", ctypes.c_int32),
                ("alpha", ctypes.c_double), ("rho", ctypes.c_double)]


SCORE_FN = ctypes.CFUNCTYPE(
    ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double))


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        i32p = ctypes.POINTER(ctypes.c_int32)
        f32p = ctypes.POINTER(ctypes.c_float)
        L.orc_digamma_table.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
        L.orc_fixed_tables.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int64)]
        L.orc_ksg_point.argtypes = [f32p, f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                    i32p, i32p, i32p, f32p, f32p, f32p]
        L.orc_ksg_window.argtypes = [f32p, f32p, ctypes.c_int64, ctypes.c_int32,
                                     i32p, i32p, i32p, f32p, f32p, f32p, ctypes.POINTER(OrcMI)]
        L.orc_ksg_window_est.argtypes = [f32p, f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                         i32p, i32p, i32p, f32p, f32p, f32p, ctypes.POINTER(OrcMI)]
        L.orc_ksg_point_est.argtypes = [f32p, f32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int64, i32p, i32p, i32p, f32p, f32p, f32p]
        L.orc_set_mutation.argtypes = [ctypes.c_int32]
        L.orc_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.orc_splitmix64_at.restype = ctypes.c_uint64
        L.orc_series_score_addr.restype = ctypes.c_void_p
        for fn in (L.orc_search_td, L.orc_search_bu):
            fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                           ctypes.POINTER(OrcParams), ctypes.POINTER(OrcWindow), ctypes.c_int64,
                           ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        L.orc_search_chunked.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.POINTER(OrcParams), ctypes.c_int32,
                                         ctypes.POINTER(OrcWindow), ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        L.orc_nscores.argtypes = [ctypes.c_double] * 5 + [ctypes.POINTER(ctypes.c_double)] * 2
        L.orc_search_auto.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.POINTER(OrcParams), ctypes.POINTER(OrcSelectParams),
                                      ctypes.POINTER(OrcWindow), ctypes.c_int64,
                                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
        _lib = L
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


class mutation:
    """Context manager that plants one of the oracle's named mistakes (tests only)."""

    def __init__(self, name: str):
        self.code = MUTATIONS[name]

    def __enter__(self):
        lib().orc_set_mutation(self.code)
        return self

    def __exit__(self, *exc):
        lib().orc_set_mutation(0)
        return False


def digamma_table(n_max: int) -> np.ndarray:
    out = np.empty(n_max + 1, dtype=np.float64)
    rc = lib().orc_digamma_table(n_max, _ptr(out, ctypes.c_double))
    assert rc == 0
    return out


def fixed_tables(n_max: int):
    psi = np.empty(n_max + 1, dtype=np.int64)
    lg = np.empty(n_max + 1, dtype=np.int64)
    rc = lib().orc_fixed_tables(n_max, _ptr(psi, ctypes.c_int64), _ptr(lg, ctypes.c_int64))
    assert rc == 0
    return psi, lg


def ksg_window(x, y, k: int, points: bool = True, estimator: int = 0):
    """KSG MI of one window (estimator 0: Kraskov's second, Eq. KSGmi; 1: Kraskov's first);
    returns a dict with the scalars and per-point arrays."""
    x = _f32(x)
    y = _f32(y)
    m = x.shape[0]
    assert y.shape[0] == m
    res = OrcMI()
    arrs = {}
    if points:
        for name, dt in (("nx", np.int32), ("ny", np.int32), ("c", np.int32),
                         ("eps", np.float32), ("dx", np.float32), ("dy", np.float32)):
            arrs[name] = np.empty(m, dtype=dt)
        ptrs = [_ptr(arrs[n], ctypes.c_int32) for n in ("nx", "ny", "c")] + \
               [_ptr(arrs[n], ctypes.c_float) for n in ("eps", "dx", "dy")]
    else:
        ptrs = [None] * 6
    rc = lib().orc_ksg_window_est(_ptr(x, ctypes.c_float), _ptr(y, ctypes.c_float), m, k,
                                  estimator, *ptrs, ctypes.byref(res))
    if rc != 0:
        raise ValueError("orc_ksg_window failed with %d (m=%d, k=%d)" % (rc, m, k))
    out = {f: getattr(res, f) for f, _ in OrcMI._fields_}
    out.update(arrs)
    return out


def ksg_point(x, y, k: int, i: int, estimator: int = 0):
    """Counts of one point i of a window (O(m)), for sampled checks of large windows."""
    x = _f32(x)
    y = _f32(y)
    vals = [ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(),
            ctypes.c_float(), ctypes.c_float(), ctypes.c_float()]
    rc = lib().orc_ksg_point_est(_ptr(x, ctypes.c_float), _ptr(y, ctypes.c_float), x.shape[0], k,
                                 estimator, i, *[ctypes.byref(v) for v in vals])
    if rc != 0:
        raise ValueError("orc_ksg_point failed with %d" % rc)
    return dict(zip(("nx", "ny", "c", "eps", "dx", "dy"), [v.value for v in vals]))


def splitmix64_at(seed: int, n: int) -> int:
    return int(lib().orc_splitmix64_at(seed & (2**64 - 1), n & (2**64 - 1)))


def make_params(k=4, score_kind=0, sigma=0.2, tau=None, s_min=32, s_max=256, delta_td=0,
                delta_bu=0, h=8, t_max_idle=3, p=3, pruning=0, max_steps=10000, seed=0,
                chunks=0):
    if tau is None:
        tau = sigma / 4.0
    return OrcParams(k, score_kind, sigma, tau, s_min, s_max, delta_td, delta_bu, h,
                     t_max_idle, p, pruning, max_steps, chunks, seed)


def _search(fn_name, score, t_begin, t_end, params):
    L = lib()
    cap = 1 << 16
    out = (OrcWindow * cap)()
    n_out = ctypes.c_int64()
    n_evals = ctypes.c_int64()
    keep = score  # keep the callback or scorer alive for the duration of the call
    if isinstance(score, tuple):          # (function pointer, user struct)
        fptr, user = score
        rc = getattr(L, fn_name)(fptr, ctypes.byref(user), t_begin, t_end, ctypes.byref(params),
                                 out, cap, ctypes.byref(n_out), ctypes.byref(n_evals))
    else:                                 # a Python callable (t_s, t_e) -> (score, mi)
        def cb(_user, ts, te, sc, mi):
            try:
                s, v = score(int(ts), int(te))
            except Exception:
                return -1
            sc[0] = s
            mi[0] = v
            return 0
        cfun = SCORE_FN(cb)
        rc = getattr(L, fn_name)(ctypes.cast(cfun, ctypes.c_void_p), None, t_begin, t_end,
                                 ctypes.byref(params), out, cap, ctypes.byref(n_out),
                                 ctypes.byref(n_evals))
    del keep
    if rc != 0:
        raise ValueError("%s failed with %d" % (fn_name, rc))
    wins = [(out[i].t_s, out[i].t_e, out[i].score, out[i].mi) for i in range(n_out.value)]
    return wins, n_evals.value


def series_scorer(x, y, k: int, score_kind: int = 0, estimator: int = 0):
    x = _f32(x)
    y = _f32(y)
    user = OrcSeriesScorer(x.ctypes.data, y.ctypes.data, x.shape[0], k, score_kind, 0, estimator, 0)
    user._keep = (x, y)
    return (ctypes.c_void_p(lib().orc_series_score_addr()), user)


def search_td(x_or_score, y=None, t_begin=0, t_end=None, estimator=0, **kw):
    """SYCOS_TD over [t_begin, t_end).  ``x_or_score`` is a series (with ``y``) or a
    callable (t_s, t_e) -> (score, mi) standing in for the window score."""
    params = make_params(**kw)
    if callable(x_or_score):
        score = x_or_score
    else:
        score = series_scorer(x_or_score, y, params.k, params.score_kind, estimator)
        if t_end is None:
            t_end = len(x_or_score)
    return _search("orc_search_td", score, t_begin, t_end, params)


def search_bu(x_or_score, y=None, t_begin=0, t_end=None, estimator=0, **kw):
    """SYCOS_BU over [t_begin, t_end); arguments as for :func:`search_td`."""
    params = make_params(**kw)
    if callable(x_or_score):
        score = x_or_score
    else:
        score = series_scorer(x_or_score, y, params.k, params.score_kind, estimator)
        if t_end is None:
            t_end = len(x_or_score)
    return _search("orc_search_bu", score, t_begin, t_end, params)


def search_chunked(x_or_score, y=None, t_begin=0, t_end=None, mode=0, chunks=2, estimator=0, **kw):
    """Algorithm 4: SYCOS_TD (mode 0) or SYCOS_BU (mode 1) on `chunks` overlapping chunks of
    [t_begin, t_end); returns (windows, n_evals) like :func:`search_td`."""
    params = make_params(chunks=chunks, **kw)
    if callable(x_or_score):
        score = x_or_score
    else:
        score = series_scorer(x_or_score, y, params.k, params.score_kind, estimator)
        if t_end is None:
            t_end = len(x_or_score)
    L = lib()
    cap = 1 << 16
    out = (OrcWindow * cap)()
    n_out = ctypes.c_int64()
    n_evals = ctypes.c_int64()
    if isinstance(score, tuple):
        fptr, user = score
        rc = L.orc_search_chunked(fptr, ctypes.byref(user), t_begin, t_end, ctypes.byref(params),
                                  mode, out, cap, ctypes.byref(n_out), ctypes.byref(n_evals))
    else:
        def cb(_user, ts, te, sc, mi):
            try:
                s_, v_ = score(int(ts), int(te))
            except Exception:
                return -1
            sc[0] = s_
            mi[0] = v_
            return 0
        cfun = SCORE_FN(cb)
        rc = L.orc_search_chunked(ctypes.cast(cfun, ctypes.c_void_p), None, t_begin, t_end,
                                  ctypes.byref(params), mode, out, cap, ctypes.byref(n_out),
                                  ctypes.byref(n_evals))
    if rc != 0:
        raise ValueError("orc_search_chunked failed with %d" % rc)
    wins = [(out[i].t_s, out[i].t_e, out[i].score, out[i].mi) for i in range(n_out.value)]
    return wins, n_evals.value


def nscores(t_td, t_bu, nl_td, ns_bu, alpha=0.5):
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().orc_nscores(t_td, t_bu, nl_td, ns_bu, alpha, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def search_auto(x_or_score, y=None, t_begin=0, t_end=None, partitions=20, samples=6, alpha=0.5,
                rho=0.5, estimator=0, **kw):
    """Algorithm 3 (iSYCOS selection) over [t_begin, t_end); returns (windows, n_evals,
    selected (0 TD / 1 BU), (nscore_TD, nscore_BU)).  Arguments as for :func:`search_td`."""
    params = make_params(**kw)
    if callable(x_or_score):
        score = x_or_score

        def cb(_user, ts, te, sc, mi):
            try:
                s, v = score(int(ts), int(te))
            except Exception:
                return -1
            sc[0] = s
            mi[0] = v
            return 0
        cfun = SCORE_FN(cb)
        fptr, user_ref = ctypes.cast(cfun, ctypes.c_void_p), None
    else:
        fptr, user = series_scorer(x_or_score, y, params.k, params.score_kind, estimator)
        user_ref = ctypes.byref(user)
        if t_end is None:
            t_end = len(x_or_score)
    sp = OrcSelectParams(partitions, samples, alpha, rho)
    cap = 1 << 16
    out = (OrcWindow * cap)()
    n_out, n_evals = ctypes.c_int64(), ctypes.c_int64()
    sel = ctypes.c_int32()
    sc = (ctypes.c_double * 2)()
    rc = lib().orc_search_auto(fptr, user_ref, t_begin, t_end, ctypes.byref(params),
                               ctypes.byref(sp), out, cap, ctypes.byref(n_out), ctypes.byref(n_evals),
                               ctypes.byref(sel), sc)
    if rc != 0:
        raise ValueError("orc_search_auto failed with %d" % rc)
    wins = [(out[i].t_s, out[i].t_e, out[i].score, out[i].mi) for i in range(n_out.value)]
    return wins, n_evals.value, sel.value, (sc[0], sc[1])
