"""The library's search machines (SYCOS_TD, SYCOS_BU, Alg. 3 selection, Alg. 4 chunks) run
on the host with window scores from the CPU oracle, against the oracle's own searches (CPU).

`tests/host_search/host_search_main.cu` links the library's search logic (`csrc/search.cu`)
with a stand-in engine that scores each window of a round with the oracle's estimator, so
the decisions, the speculation and caching of the machines and the batching of a round are
checked without a GPU: the found windows must be the oracle's, bit for bit, and the number
of window scores the decisions read must equal the oracle's evaluation count.  The MI
kernels are covered by the GPU tests.
"""
from __future__ import annotations

import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2204_09131_gb300 import synth
from tests import _search_pins

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "host_search", "host_search_main.cu")
BUILD = os.path.join(HERE, "host_search", "_build")
EXE = os.path.join(BUILD, "host_search")


@pytest.fixture(scope="module")
def driver():
    from paper_2204_09131_gb300 import build as B
    try:
        nvcc = B.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    os.makedirs(BUILD, exist_ok=True)
    obj = os.path.join(BUILD, "oracle.o")
    subprocess.run(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-std=c11", "-c",
                    os.path.join(ROOT, "oracle", "isycos_oracle.c"), "-o", obj], check=True)
    subprocess.run([nvcc, *B.ARCH, "-O2", "-std=c++17", "--expt-relaxed-constexpr",
                    "-I" + B.INCLUDE, "-I" + B.CSRC, SRC, os.path.join(B.CSRC, "search.cu"), obj,
                    "-o", EXE, "-lm"], check=True, capture_output=True)
    return EXE


def _series_file(tmp_path, pairs):
    n = len(pairs[0][0])
    path = os.path.join(str(tmp_path), "series.bin")
    with open(path, "wb") as f:
        np.array([len(pairs)], np.int32).tofile(f)
        np.array([n], np.int64).tofile(f)
        for x, y in pairs:
            np.asarray(x, np.float32).tofile(f)
            np.asarray(y, np.float32).tofile(f)
    return path


def _run(exe, path, **kw):
    args = [exe, path] + ["%s=%s" % (k, v) for k, v in kw.items()]
    out = subprocess.run(args, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    res, cur = [], None
    for line in out.stdout.splitlines():
        f = line.split()
        if f[0] == "M":
            cur = {"decided": int(f[3]), "found": []}
            res.append(cur)
        elif f[0] == "W":
            cur["found"].append((int(f[1]), int(f[2]), float(f[3]), float(f[4])))
    return res


def _same(got, ref, n_ref):
    assert [(a, b) for a, b, _, _ in got["found"]] == [(a, b) for a, b, _, _ in ref]
    for (_, _, s, m), (_, _, rs, rm) in zip(got["found"], ref):
        assert s == rs and m == rm
    assert got["decided"] == n_ref


@pytest.fixture(scope="module")
def pairs():
    x0, y0 = synth.planted_small_pair()
    x1, y1, _ = synth.planted_pair(6, 3, len(x0))
    return [(x0, y0), (x1, y1)]


ORC_KEYS = ("k", "score_kind", "sigma", "tau", "s_min", "s_max", "delta_td", "delta_bu", "h",
            "t_max_idle", "p", "pruning", "max_steps", "seed")

CASES = [
    # SYCOS_TD: pruning off / on, raw-MI scores, an explicit step that leaves the grid
    dict(mode=0, pruning=0),
    dict(mode=0, pruning=1),
    dict(mode=0, pruning=1, score_kind=1, sigma=0.5, tau=0.1),
    dict(mode=0, pruning=1, delta_td=7),
    # SYCOS_BU: pruning off / on, seeds, idle limits, a step that does not divide s_min
    dict(mode=1, pruning=0, seed=3),
    dict(mode=1, pruning=1, seed=31),
    dict(mode=1, pruning=1, score_kind=1, sigma=0.5, tau=0.1, seed=5),
    dict(mode=1, pruning=1, t_max_idle=1, seed=7),
    dict(mode=1, pruning=1, t_max_idle=5, h=3, seed=8),
    dict(mode=1, pruning=1, t_max_idle=10, seed=12),   # rings beyond 8 share cache slots
    dict(mode=1, pruning=1, delta_bu=5, seed=9),
    # the second estimator's counterpart (Kraskov's first)
    dict(mode=0, pruning=1, estimator=1),
    dict(mode=1, pruning=1, estimator=1, seed=11),
]


@pytest.mark.parametrize("kw", CASES)
def test_machines_match_oracle(driver, tmp_path, pairs, kw):
    path = _series_file(tmp_path, pairs)
    got = _run(driver, path, s_max=256, **kw)
    okw = {k: v for k, v in kw.items() if k in ORC_KEYS}
    for (x, y), g in zip(pairs, got):
        ref, n = (O.search_td if kw["mode"] == 0 else O.search_bu)(
            x, y, s_max=256, estimator=kw.get("estimator", 0), **okw)
        _same(g, ref, n)


@pytest.mark.parametrize("spec,incremental", [(0, 1), (1, 1), (24, 0), (64, 2)])
def test_bu_speculation_and_chains_change_work_not_results(driver, tmp_path, pairs, spec,
                                                            incremental):
    """Climbs asked ahead, extension windows asked ahead and incremental chains change the
    rounds, never the decisions."""
    path = _series_file(tmp_path, pairs)
    kw = dict(mode=1, pruning=1, seed=31)
    got = _run(driver, path, s_max=256, spec=spec, incremental=incremental, **kw)
    okw = {k: v for k, v in kw.items() if k != "mode"}
    for (x, y), g in zip(pairs, got):
        ref, n = O.search_bu(x, y, s_max=256, **okw)
        _same(g, ref, n)


def test_sub_range(driver, tmp_path, pairs):
    path = _series_file(tmp_path, pairs)
    for mode in (0, 1):
        got = _run(driver, path, s_max=128, mode=mode, pruning=1, t_begin=300, t_end=1700)
        for (x, y), g in zip(pairs, got):
            ref, n = (O.search_td if mode == 0 else O.search_bu)(
                x, y, t_begin=300, t_end=1700, s_max=128, pruning=1)
            _same(g, ref, n)


@pytest.mark.parametrize("mode", [0, 1])
def test_chunked_matches_oracle(driver, tmp_path, pairs, mode):
    """Algorithm 4: three overlapping chunks searched independently."""
    path = _series_file(tmp_path, pairs)
    got = _run(driver, path, s_max=128, mode=mode, pruning=1, chunks=3)
    for (x, y), g in zip(pairs, got):
        ref, n = O.search_chunked(x, y, mode=mode, chunks=3, s_max=128, pruning=1)
        _same(g, ref, n)


def test_selection_matches_oracle(driver, tmp_path, pairs):
    """Algorithm 3: sampled partitions searched with both algorithms, then the choice."""
    path = _series_file(tmp_path, pairs)
    got = _run(driver, path, s_max=128, mode=2, pruning=1, sel_partitions=8, sel_samples=3)
    for (x, y), g in zip(pairs, got):
        ref, n, _, _ = O.search_auto(x, y, partitions=8, samples=3, s_max=128, pruning=1)
        _same(g, ref, n)


def _table_case(tmp_path, case, spec):
    """The series file (zeros) and harness arguments of a hand-traced case in table mode."""
    _, search, score, t_end, kw, _ = case
    zeros = np.zeros(t_end, np.float32)
    series = _series_file(tmp_path, [(zeros, zeros)])
    table = os.path.join(str(tmp_path), "table.txt")
    with open(table, "w") as f:
        for ts in range(t_end):
            for te in range(ts, t_end):
                f.write("%d %d %.17g\n" % (ts, te, score(ts, te)))
    args = dict(table=table, t_end=t_end, spec=spec)
    rename = dict(partitions="sel_partitions", samples="sel_samples", alpha="sel_alpha", rho="sel_rho")
    for key, v in kw.items():
        args[rename.get(key, key)] = v
    args.setdefault("mode", {"td": 0, "bu": 1, "auto": 2}.get(search, 0))
    return series, args


@pytest.mark.parametrize("spec", [0, 24, 64])
@pytest.mark.parametrize("case", _search_pins.machine_cases(), ids=lambda c: c[0])
def test_machines_follow_the_hand_traces(driver, tmp_path, case, spec):
    """The library's search machines on the hand-traced score tables of tests/_search_pins.py
    (every window of the range listed with its score), with 0, 24 and 64 BU climbs asked
    ahead: the hand-traced windows, and the oracle's decided-window count."""
    name, search, score, t_end, kw, expect = case
    series, args = _table_case(tmp_path, case, spec)
    got = _run(driver, series, **args)[0]
    assert [(a, b) for a, b, _, _ in got["found"]] == expect, (name, got["found"])
    ref, n = _search_pins.oracle_run(search, score, t_end, kw)
    _same(got, ref, n)


def test_launch_layout_invariants():
    """The launch layout shared by the host runtime and the batched MI kernel (size buckets,
    warps per item, bucket tables, grid size, shared-memory sizes) satisfies its invariants
    (`tests/host_search/layout_main.cu`)."""
    from paper_2204_09131_gb300 import build as B
    try:
        nvcc = B.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    os.makedirs(BUILD, exist_ok=True)
    exe = os.path.join(BUILD, "layout")
    subprocess.run([nvcc, *B.ARCH, "-O2", "-std=c++17", "--expt-relaxed-constexpr",
                    "-I" + B.INCLUDE, "-I" + B.CSRC, os.path.join(HERE, "host_search", "layout_main.cu"),
                    "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout[-2000:]


@pytest.mark.parametrize("seed", range(8))
def test_random_configurations(driver, tmp_path, pairs, seed):
    """Seeded random parameter sets and sub-ranges (k, window sizes, steps, idle limits,
    noise thresholds): every window a machine asks for lies inside the range (the stand-in
    engine rejects any other) and the decisions are the oracle's."""
    rng = np.random.default_rng(1000 + seed)
    k = int(rng.choice([2, 3, 4, 6]))
    s_min = int(rng.choice([16, 24, 32, 40]))
    s_max = int(rng.choice([s_min * 2, s_min * 4, 192, 256]))
    s_max = max(s_max, s_min)
    n = len(pairs[0][0])
    t_begin = int(rng.integers(0, 400))
    t_end = int(rng.integers(n - 400, n + 1))
    kw = dict(k=k, s_min=s_min, s_max=s_max, pruning=int(rng.integers(0, 2)),
              delta_bu=int(rng.choice([0, 3, 4, 7])), delta_td=int(rng.choice([0, 0, 5, 9])),
              t_max_idle=int(rng.choice([1, 2, 3, 6])), h=int(rng.choice([4, 8, 12])),
              sigma=float(rng.choice([0.15, 0.2, 0.3])), seed=int(rng.integers(0, 1 << 30)))
    est = int(rng.integers(0, 4) == 0)   # Kraskov's first estimator in a quarter of them
    path = _series_file(tmp_path, pairs)
    for mode in (0, 1):
        got = _run(driver, path, mode=mode, t_begin=t_begin, t_end=t_end, estimator=est,
                   spec=int(rng.choice([0, 5, 24])), **kw)
        for (x, y), g in zip(pairs, got):
            ref, n_ref = (O.search_td if mode == 0 else O.search_bu)(
                x, y, t_begin=t_begin, t_end=t_end, estimator=est, **kw)
            _same(g, ref, n_ref)


def _serve_queries(rng, n_queries, n):
    qs = []
    for i in range(n_queries):
        qs.append(dict(pair=i % 2, mode=int(rng.integers(0, 2)), tb=int(rng.integers(0, 300)),
                       te=int(rng.integers(n - 300, n + 1)), k=int(rng.choice([3, 4])), s_min=32,
                       s_max=int(rng.choice([128, 256])), pruning=int(rng.integers(0, 2)),
                       seed=int(rng.integers(0, 1 << 30)), est=int(rng.integers(0, 4) == 0),
                       cancel=int(i == 5)))
    return qs


def _check_served(exe, tmp_path, pairs, seed, batch=False):
    rng = np.random.default_rng(seed)
    qs = _serve_queries(rng, 14, len(pairs[0][0]))
    series = _series_file(tmp_path, pairs)
    qfile = os.path.join(str(tmp_path), "queries.txt")
    with open(qfile, "w") as f:
        for q in qs:
            f.write("%d %d %d %d %d %d %d %d %d %d %d\n" % (
                q["pair"], q["mode"], q["tb"], q["te"], q["k"], q["s_min"], q["s_max"],
                q["pruning"], q["seed"], q["est"], q["cancel"]))
    out = subprocess.run([exe, series, qfile] + (["batch"] if batch else []), capture_output=True,
                         text=True, timeout=900)
    if "FATAL: ThreadSanitizer" in out.stderr:   # the sanitizer cannot start on this system
        pytest.skip(out.stderr.strip().splitlines()[0][:200])
    assert out.returncode == 0, (out.stdout[-500:], out.stderr[-3000:])
    for report in ("ThreadSanitizer", "AddressSanitizer", "runtime error"):
        assert report not in out.stderr, out.stderr[-3000:]
    res, cur = {}, None
    for line in out.stdout.splitlines():
        f = line.split()
        if f[0] == "Q":
            cur = int(f[1])
            res[cur] = (int(f[2]), [])
        elif f[0] == "W":
            res[cur][1].append((int(f[1]), int(f[2]), float(f[3]), float(f[4])))
    assert sorted(res) == list(range(len(qs)))
    for i, q in enumerate(qs):
        st, got = res[i]
        if q["cancel"] and st != 0 and not batch:
            continue   # cancelled before it finished
        assert st == 0, (i, st)
        x, y = pairs[q["pair"]]
        ref, _ = (O.search_td if q["mode"] == 0 else O.search_bu)(
            x, y, t_begin=q["tb"], t_end=q["te"], k=q["k"], s_min=q["s_min"], s_max=q["s_max"],
            pruning=q["pruning"], seed=q["seed"], estimator=q["est"])
        assert got == list(ref), i


_SERVE_BUILDS = {}
_SANITIZERS = {"": [], "tsan": ["-fsanitize=thread"],
               "asan": ["-fsanitize=address", "-fsanitize=undefined", "-fno-omit-frame-pointer"]}


def _build_serve(flavour):
    if flavour not in _SERVE_BUILDS:   # built once per session and flavour
        _SERVE_BUILDS[flavour] = _build_serve_now(flavour)
    return _SERVE_BUILDS[flavour]


def _build_serve_now(flavour):
    from paper_2204_09131_gb300 import build as B
    try:
        nvcc = B.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    os.makedirs(BUILD, exist_ok=True)
    tag = "_" + flavour if flavour else ""
    flags = _SANITIZERS[flavour]

    def failed(what, err):
        if flavour:   # the sanitizer may be missing here: skip rather than fail
            pytest.skip("cannot build with %s (%s): %s" % (flavour, what, err[-200:]))
        raise AssertionError(err[-2000:])

    objs = []
    for src in (os.path.join(HERE, "host_search", "host_serve_main.cu"), os.path.join(B.CSRC, "serve.cu"),
                os.path.join(B.CSRC, "search.cu")):
        obj = os.path.join(BUILD, "serve%s_%s.o" % (tag, os.path.basename(src)[:-3]))
        cmd = [nvcc, *B.ARCH, "-O1", "-g", "-std=c++17", "--expt-relaxed-constexpr",
               "-I" + B.INCLUDE, "-I" + B.CSRC, "-c", src, "-o", obj]
        for flag in flags:
            cmd += ["-Xcompiler", flag]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            failed("compile", r.stderr)
        objs.append(obj)
    orc = os.path.join(BUILD, "oracle%s.o" % tag)
    r = subprocess.run(["gcc", "-O1", "-g", *flags, "-fno-fast-math", "-ffp-contract=off", "-std=c11",
                        "-c", os.path.join(ROOT, "oracle", "isycos_oracle.c"), "-o", orc],
                       capture_output=True, text=True)
    if r.returncode != 0:
        failed("compile", r.stderr)
    exe = os.path.join(BUILD, "host_serve%s" % tag)
    cudalib = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64")
    link = subprocess.run(["g++", *[f for f in flags if f.startswith("-fsanitize")], *objs, orc, "-o", exe,
                           "-L" + cudalib, "-lcudart_static", "-ldl", "-lpthread", "-lrt", "-lm"],
                          capture_output=True, text=True)
    if link.returncode != 0:
        failed("link", link.stderr)
    return exe


def test_served_queries_match_oracle(tmp_path, pairs):
    """The serving loop (csrc/serve.cu: admission with fewer slots than queries, four worker
    lanes, submissions from two threads, a cancellation) returns every query's own search."""
    _check_served(_build_serve(""), tmp_path, pairs, 21)


def test_serving_threads_race_free(tmp_path, pairs):
    """The same under ThreadSanitizer: the server's threads, the submitting threads and the
    pollers share no unsynchronised state."""
    _check_served(_build_serve("tsan"), tmp_path, pairs, 22)


def test_search_queries_lanes_match_oracle_race_free(tmp_path, pairs):
    """isycos_search_queries with TD and BU queries in one call (engine lanes on host threads,
    TD lanes apart) under ThreadSanitizer: every query's windows are its own search's."""
    _check_served(_build_serve("tsan"), tmp_path, pairs, 23, batch=True)


def test_serving_memory_safe(tmp_path, pairs):
    """The serving loop and isycos_search_queries under AddressSanitizer and
    UndefinedBehaviorSanitizer: no invalid access, leak or undefined behaviour in admission,
    the worker lanes, cancellation or the batched call, and every result still the oracle's."""
    exe = _build_serve("asan")
    _check_served(exe, tmp_path, pairs, 24)
    _check_served(exe, tmp_path, pairs, 25, batch=True)


def test_search_machines_memory_safe(tmp_path, pairs):
    """The search machines under AddressSanitizer and UndefinedBehaviorSanitizer: no invalid
    access and no undefined behaviour in TD, BU (speculation off and at 64 climbs, a step that
    leaves the lattice, long idle limits), selection or chunks, and the oracle's windows."""
    from paper_2204_09131_gb300 import build as B
    try:
        nvcc = B.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    os.makedirs(BUILD, exist_ok=True)
    san = ["-fsanitize=address", "-fsanitize=undefined", "-fno-omit-frame-pointer"]
    objs = []
    for src in (SRC, os.path.join(B.CSRC, "search.cu")):
        obj = os.path.join(BUILD, "asan_%s.o" % os.path.basename(src)[:-3])
        cmd = [nvcc, *B.ARCH, "-O1", "-g", "-std=c++17", "--expt-relaxed-constexpr", "-I" + B.INCLUDE,
               "-I" + B.CSRC, "-c", src, "-o", obj]
        for flag in san:
            cmd += ["-Xcompiler", flag]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            pytest.skip("cannot build with the sanitizers: " + r.stderr[-200:])
        objs.append(obj)
    orc = os.path.join(BUILD, "asan_oracle.o")
    r = subprocess.run(["gcc", "-O1", "-g", *san, "-fno-fast-math", "-ffp-contract=off", "-std=c11", "-c",
                        os.path.join(ROOT, "oracle", "isycos_oracle.c"), "-o", orc], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("cannot build with the sanitizers: " + r.stderr[-200:])
    exe = os.path.join(BUILD, "host_search_asan")
    cudalib = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64")
    r = subprocess.run(["g++", "-fsanitize=address", "-fsanitize=undefined", *objs, orc, "-o", exe,
                        "-L" + cudalib, "-lcudart_static", "-ldl", "-lpthread", "-lrt", "-lm"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("no sanitizer runtime: " + r.stderr[-200:])
    path = _series_file(tmp_path, pairs)
    cases = [dict(mode=1, pruning=1, seed=31, spec=0, incremental=2),
             dict(mode=1, pruning=1, seed=10, spec=64, t_begin=300, t_end=1700),
             dict(mode=1, pruning=1, delta_bu=5, t_max_idle=10, seed=4),
             dict(mode=0, pruning=1, delta_td=7, estimator=1),
             dict(mode=2, pruning=1, sel_partitions=6, sel_samples=2, s_max=128),
             dict(mode=1, pruning=1, chunks=3, s_max=128)]
    for kw in cases:
        args = [exe, path] + ["%s=%s" % kv for kv in kw.items()]
        if "s_max" not in kw:
            args.append("s_max=256")
        out = subprocess.run(args, capture_output=True, text=True, timeout=900)
        assert "AddressSanitizer" not in out.stderr and "runtime error" not in out.stderr, out.stderr[-3000:]
        assert out.returncode == 0, (kw, out.stderr[-2000:])
    # two hand-traced cases in table mode: BU with pruning and 64 climbs ahead, the selection
    for case in _search_pins.machine_cases():
        if case[0] not in ("bu_noise_run_resets", "selection_td"):
            continue
        series, kw = _table_case(tmp_path, case, 64)
        out = subprocess.run([exe, series] + ["%s=%s" % kv for kv in kw.items()], capture_output=True,
                             text=True, timeout=900)
        assert "AddressSanitizer" not in out.stderr and "runtime error" not in out.stderr, out.stderr[-3000:]
        assert out.returncode == 0, (case[0], out.stderr[-2000:])
