"""Oracle work for the large parity tests, run in a process pool (spawned workers).

Each job regenerates its seeded series from ``synth`` (no large arrays cross the process
boundary) and calls only the oracle, so the expected values of the GPU tests never come
from the CUDA path.  The pool uses the ``spawn`` start method: workers never inherit a CUDA
context.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def series(spec):
    """(x, y) of a workload spec: ("planted", cfg, pair, n), ("tied", pair, n) or
    ("mixed", cfg, pair, n) (mixed-noise background, segments of 100..10,000 samples)."""
    from paper_2204_09131_gb300 import synth
    kind = spec[0]
    if kind == "planted":
        x, y, _ = synth.planted_pair(spec[1], spec[2], spec[3])
    elif kind == "tied":
        x, y, _ = synth.tied_pair(spec[1], spec[2])
    elif kind == "mixed":
        x, y, _ = synth.planted_pair(spec[1], spec[2], spec[3], len_lo=100, len_hi=10000,
                                     background="mixed")
    else:
        raise ValueError(kind)
    return x, y


def search_job(job):
    """job = (mode, spec, t_begin, t_end, params): the oracle's SYCOS_TD (mode 0) or SYCOS_BU
    (mode 1) on [t_begin, t_end); returns (windows, evaluated-window count)."""
    from oracle import oracle as O
    mode, spec, t0, t1, prm = job
    x, y = series(spec)
    fn = O.search_td if mode == 0 else O.search_bu
    wins, n = fn(x, y, t_begin=t0, t_end=t1, **prm)
    return [(int(a), int(b), float(s), float(m)) for a, b, s, m in wins], int(n)


def windows_job(job):
    """job = (spec, k, [(start, m), ...]): per window (s_psi, s_log, mi, h_w, nmi)."""
    from oracle import oracle as O
    spec, k, wins = job
    x, y = series(spec)
    out = []
    for s, m in wins:
        r = O.ksg_window(x[s:s + m], y[s:s + m], k, points=False)
        out.append((int(r["s_psi"]), int(r["s_log"]), r["mi"], r["h_w"], r["nmi"]))
    return out


def points_job(job):
    """job = (spec, k, start, m, [i, ...]): (n_x, n_y, c) of the listed points of one window."""
    from oracle import oracle as O
    spec, k, s, m, pts = job
    x, y = series(spec)
    xx, yy = x[s:s + m], y[s:s + m]
    out = []
    for i in pts:
        r = O.ksg_point(xx, yy, k, int(i))
        out.append((int(r["nx"]), int(r["ny"]), int(r["c"])))
    return out


def pool_map(fn, jobs):
    """Map over a spawned pool of up to 16 workers (results in job order)."""
    from oracle import oracle as O
    O.build()   # compile once before the workers load it
    n = max(1, min(16, os.cpu_count() or 1, len(jobs)))
    if n == 1:
        return [fn(j) for j in jobs]
    with mp.get_context("spawn").Pool(n) as p:
        return p.map(fn, jobs, chunksize=1)


def stratified_windows(k, n, per_bucket, big_per_bucket, seed):
    """Window sizes stratified over every size bucket b = 3 .. 14 (2^(b-1) < m <= 2^b, at
    least k + 1 points): per_bucket windows for b <= 12, big_per_bucket for b = 13, 14; starts
    uniform.  Returns a list of (start, m)."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(3, 15):
        lo, hi = max(k + 1, (1 << (b - 1)) + 1), 1 << b
        if lo > hi:
            continue
        cnt = per_bucket if b <= 12 else big_per_bucket
        for _ in range(cnt):
            m = int(rng.integers(lo, hi + 1))
            out.append((int(rng.integers(0, n - m + 1)), m))
    return out
