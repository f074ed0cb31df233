"""Benchmark: window-MI evaluations per second of the iSYCOS hot path on GB300.

Workload (one "step"): the paper's searches over 64 synthetic pairs of FP32 series of length
100,000 with planted linear / quadratic / sin(3X) / exp(X) segments (lengths log-uniform in
[50, 5000], SNR in {0.5, 2, 10}, iid N(0,1) background), k = 4, window sizes 32-4096,
sigma = 0.2 on the normalised score, noise pruning on: a SYCOS_TD (Algorithm 1) and a
SYCOS_BU (Algorithm 2) query per pair, 128 queries run concurrently on the library's engine
lanes, each lane merging its queries' window frontiers into persistent, size-bucketed MI
launches.  The series stay resident in HBM (value); the e2e figure uploads them from pinned
host memory and reads the found windows back inside the timed region.

One JSON line per run.  Its roofline counts the lane operations of the work the MI kernels
did (their work counters: brute-force evaluations, the sorted path's scan visits, search steps
and sort compare-exchanges, each at a stated cost) over the union of the MI kernel's launch
intervals, against 152 SMs x 4 warp instructions per clock x 32 lanes at the sampled SM
clock; the brute-force-equivalent figure (11 lane operations per ordered pair m (m - 1) of
every evaluated window) is reported beside it, labelled.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "window-MI evals/sec and pairwise comparisons/sec vs FP32 roofline; p50/p99 query latency"
N_PAIRS = 64
N_LEN = 100_000
PARAMS = dict(k=4, s_min=32, s_max=4096, sigma=0.2, tau=0.05, pruning=1, seed=20220419)
# lane operations per ordered pair of the brute-force method: pass 1 (two subtractions with
# |.|, max, compare) = 5 with the predicated insertion, pass 2 (two subtractions, two
# compares, two adds) = 6
OPS_PER_PAIR = 11
# lane operations per unit of the work counters (isycos_stats work_*): a brute-force point x
# candidate evaluation (both passes, as above); an outward-scan visit of the sorted path (a
# broadcast load, two subtractions with |.|, max, compare with the list's last entry and the
# index tie-break); a binary-search or duplicate-scan step (load, subtraction with |.|,
# compare, two selects); a bitonic compare-exchange (64-bit compare, two selects, exchange)
OPS_PER_UNIT = {"work_bf": 11, "work_scan": 6, "work_search": 5, "work_sort": 4}


def method_ops(st):
    """Lane operations of the work the MI kernels did (work counters x cost per unit)."""
    return sum(OPS_PER_UNIT[f] * st[f] for f in OPS_PER_UNIT)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--pairs", type=int, default=N_PAIRS)
    ap.add_argument("--length", type=int, default=N_LEN)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-stress", action="store_true", help="skip the noise-pruning stress case")
    ap.add_argument("--stress-case", action="store_true",
                    help="run only the noise-pruning stress case and print its JSON")
    ap.add_argument("--stress-pairs", type=int, default=256)
    ap.add_argument("--stress-length", type=int, default=200_000)
    ap.add_argument("--kernel-case", default=None,
                    help="time one MI batch instead of the searches: td4096, td1024, td256, "
                         "ring (BU-ring sized windows), mix (all TD layers)")
    ap.add_argument("--case-pairs", type=int, default=8)
    ap.add_argument("--search-case", default=None, choices=["td", "bu", "mix", "select", "chunked"],
                    help="time one kind of search query over --case-pairs pairs of --length "
                         "points instead of the default step (per-size launch statistics)")
    ap.add_argument("--lanes", type=int, default=0, help="ISYCOS_OPT_LANES (0: library default)")
    ap.add_argument("--serving-case", action="store_true",
                    help="the served form at scale: --serve-series resident series of "
                         "--serve-length points, Poisson streams of --serve-queries queries at "
                         "fractions --serve-rates of a measured capacity (p50/p99 latency)")
    ap.add_argument("--serve-series", type=int, default=512)
    ap.add_argument("--serve-length", type=int, default=1_000_000)
    ap.add_argument("--serve-queries", type=int, default=400)
    ap.add_argument("--serve-calibrate", type=int, default=256,
                    help="served form in the default run: queries submitted at once to measure capacity")
    ap.add_argument("--serve-stream", type=int, default=2000,
                    help="served form in the default run: queries of the Poisson stream")
    ap.add_argument("--serve-rates", default="0.3,0.7,1.0,1.3")
    ap.add_argument("--speculation", type=int, default=-1,
                    help="ISYCOS_OPT_SPECULATION (BU climbs asked ahead; -1: library default)")
    ap.add_argument("--plain", action="store_true", help="also time the one-window-per-launch form")
    ap.add_argument("--kernel-opt", type=int, default=0,
                    help="ISYCOS_OPT_KERNEL: 0 auto, 1 brute force only, 2 sorted path")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_pairs(rank, n_pairs, length, world=1):
    """This rank's pairs: every world-th of world * n_pairs pairs (weak scaling, no collective
    on the data path)."""
    from paper_2204_09131_gb300 import shard, synth
    pairs = []
    for p in shard.shard_indices(world * n_pairs, rank, world):
        x, y, _ = synth.planted_pair(2, p, length)
        pairs.append((x, y))
    return pairs


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([s.strip() for s in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for i, nm in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


def run_step(api, ctx, ids, length):
    """SYCOS_TD and SYCOS_BU queries of every pair in one call: independent queries whose
    frontiers run concurrently on the engine lanes and share the GPU."""
    queries = [(a, b, 0, length, dict(PARAMS, mode=mode)) for mode in (0, 1) for a, b in ids]
    res = api.isycos_search_queries(ctx, queries)
    return sum(len(r) for r in res)


def flush_l2(torch, buf):
    buf.fill_(1.0)          # 256 MiB write, larger than the 129 MB L2


def _serving_pair(job):
    """One resident pair of the served workload (config-4 shape); run in a spawned worker."""
    p, length = job
    from paper_2204_09131_gb300 import synth
    x, y, _ = synth.planted_pair(4, p, length)
    return x, y


def put_serving_series(api, ctx, n_pairs, length):
    """Generate the served pairs in a spawned pool (no CUDA in the workers) and make them
    resident as they arrive; returns the pairs' series ids."""
    import multiprocessing as mp
    ids = []
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        for x, y in pool.imap(_serving_pair, [(p, length) for p in range(n_pairs)], chunksize=2):
            ids.append((api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)))
    return ids


def serving_queries(ids, length, n, seed):
    """Random queries over the resident pairs: a random pair, a range log-uniform in
    [1e3, length], s_max a power of two log-uniform in [256, 16384] clipped to range / 2,
    SYCOS_TD and SYCOS_BU alternating."""
    rng = np.random.default_rng(seed)
    qs = []
    for i in range(n):
        a, b = ids[int(rng.integers(0, len(ids)))]
        span = int(np.exp(rng.uniform(np.log(1000), np.log(length))))
        lo = int(rng.integers(0, length - span + 1))
        s_max = int(2 ** rng.integers(8, 15))
        s_max = max(64, min(s_max, span // 2))
        qs.append((a, b, lo, lo + span, dict(PARAMS, s_max=s_max, mode=int(i % 2))))
    return qs


def serve_stream(api, ctx, qs, gaps):
    """Submit the queries at the given inter-arrival gaps (seconds) while polling the pending
    ones; returns latencies and admission waits (ms) and the wall time."""
    pending, lat, wait = [], {}, {}
    start = time.perf_counter()
    nxt = start

    def drain():
        still = []
        for t in pending:
            r = api.isycos_serve_poll_ex(ctx, t)
            if r is None:
                still.append(t)
            else:
                lat[t], wait[t] = r[1], r[2]
        pending[:] = still

    for q, g in zip(qs, gaps):
        nxt += g
        while time.perf_counter() < nxt:
            drain()
            time.sleep(0.0002)
        pending.append(api.isycos_serve_submit(ctx, *q[:4], q[4]))
    while pending:
        drain()
        time.sleep(0.0005)
    wall = time.perf_counter() - start
    return np.array(list(lat.values())), np.array(list(wait.values())), wall


def serving_config4(args):
    """The served form at config-4 shape: 512 resident series of 1,000,000 points (256 pairs
    with planted segments), capacity calibrated by submitting a batch of queries at once, then
    a Poisson stream at 0.7 x that capacity; p50 / p99 latency, throughput and admission wait."""
    from paper_2204_09131_gb300 import api
    n_pairs, length = args.serve_series // 2, args.serve_length
    ctx = api.isycos_create(0, 0)
    try:
        t0 = time.perf_counter()
        ids = put_serving_series(api, ctx, n_pairs, length)
        t_put = time.perf_counter() - t0
        api.isycos_autotune(ctx, PARAMS["k"])
        cal_q = serving_queries(ids, length, args.serve_calibrate, 1)
        lat_c, _, wall_c = serve_stream(api, ctx, cal_q, [0.0] * len(cal_q))
        capacity = len(cal_q) / wall_c
        qs = serving_queries(ids, length, args.serve_stream, 2)
        rate = 0.7 * capacity
        gaps = np.random.default_rng(7).exponential(1.0 / rate, len(qs))
        lat, wait, wall = serve_stream(api, ctx, qs, gaps)
        st = api.isycos_get_stats(ctx)
        return {"workload": "%d resident series x %d points (%d planted pairs); queries: a random "
                            "pair, range log-uniform 1e3-%d, s_max log-uniform 256-16384 clipped to "
                            "range/2, SYCOS_TD and SYCOS_BU alternating" % (2 * n_pairs, length, n_pairs, length),
                "resident_bytes": int(8 * n_pairs * length), "upload_s": round(t_put, 1),
                "calibration": {"queries": len(cal_q), "submitted": "all at once",
                                "capacity_qps": round(capacity, 2),
                                "p50_ms": round(float(np.percentile(lat_c, 50)), 2)},
                "queries": len(qs), "arrival": "Poisson at 0.7 x capacity",
                "arrival_rate_hz": round(rate, 2),
                "p50_ms": round(float(np.percentile(lat, 50)), 2),
                "p99_ms": round(float(np.percentile(lat, 99)), 2),
                "throughput_qps": round(len(qs) / wall, 2),
                "admission_wait_p50_ms": round(float(np.percentile(wait, 50)), 3),
                "admission_wait_p99_ms": round(float(np.percentile(wait, 99)), 3),
                "queries_done": st["queries_done"]}
    finally:
        api.isycos_destroy(ctx)


def _stress_pair(job):
    """One pair of the noise-pruning stress workload (config-3 shape); run in a spawned worker."""
    p, length = job
    from paper_2204_09131_gb300 import synth
    x, y, _ = synth.planted_pair(3, p, length, len_lo=100, len_hi=10000, background="mixed")
    return x, y


def overlap_agreement(ref, got):
    """Windows of `ref` that overlap some window of `got` (the paper's accuracy measure of the
    noise pruning: two windows count as the same when their index ranges overlap)."""
    hit = 0
    j = 0
    got = sorted((int(a), int(b)) for a, b in zip(got["t_s"], got["t_e"]))
    for a, b in sorted((int(a), int(b)) for a, b in zip(ref["t_s"], ref["t_e"])):
        while j < len(got) and got[j][1] < a:
            j += 1
        if j < len(got) and got[j][0] <= b:
            hit += 1
    return hit


def pruning_stress(args):
    """Noise-pruning stress (config-3 shape): --stress-pairs pairs of --stress-length points,
    70 % independent Gaussian / uniform / Laplace noise and 30 % planted segments of
    100-10,000 samples; SYCOS_TD and SYCOS_BU of every pair with pruning off and on (k = 4,
    window sizes 32-8192).  Per mode: decided window-MI evals/s; and the share of the windows
    found without pruning that overlap a window found with it."""
    import multiprocessing as mp
    import torch
    from paper_2204_09131_gb300 import api
    n_pairs, length = args.stress_pairs, args.stress_length
    ctx = api.isycos_create(0, 0)
    try:
        ids = []
        with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
            for x, y in pool.imap(_stress_pair, [(p, length) for p in range(n_pairs)], chunksize=2):
                ids.append((api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)))
        api.isycos_autotune(ctx, PARAMS["k"])
        base = dict(PARAMS, s_max=8192)
        out = {"workload": "%d pairs x %d points, 70%% independent noise (Gaussian / uniform / Laplace "
                           "per gap), 30%% planted segments of 100-10000 samples; k=4, sizes 32-8192"
                           % (n_pairs, length)}
        res = {}
        warm = [(a, b, 0, length, dict(base, mode=m, pruning=1)) for a, b in ids[:4] for m in (0, 1)]
        api.isycos_search_queries(ctx, warm)
        for pr in (0, 1):
            qs = [(a, b, 0, length, dict(base, mode=m, pruning=pr)) for m in (0, 1) for a, b in ids]
            torch.cuda.synchronize()
            api.isycos_reset_stats(ctx)
            t0 = time.perf_counter()
            res[pr] = api.isycos_search_queries(ctx, qs)
            dt = time.perf_counter() - t0
            st = api.isycos_get_stats(ctx)
            out["pruning_%s" % ("on" if pr else "off")] = {
                "s": round(dt, 3), "decided_windows": st["decided_windows"],
                "evals_per_s": round(st["decided_windows"] / dt, 1),
                "gpu_windows": st["windows"], "found": int(sum(len(r) for r in res[pr]))}
        for name, sl in (("td", slice(0, n_pairs)), ("bu", slice(n_pairs, 2 * n_pairs))):
            ref = res[0][sl]
            hit = sum(overlap_agreement(r, g) for r, g in zip(ref, res[1][sl]))
            tot = sum(len(r) for r in ref)
            out["agreement_" + name] = {"found_without_pruning": tot, "overlapped_with_pruning": hit,
                                        "fraction": round(hit / tot, 4) if tot else None}
        out["speedup_of_pruning"] = round(out["pruning_off"]["s"] / out["pruning_on"]["s"], 2)
        return out
    finally:
        api.isycos_destroy(ctx)


def host_info():
    """The host the oracle runs on: cores it may use and the CPU model."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = os.cpu_count()
    return {"nproc": os.cpu_count(), "usable_cores": usable,
            "cpu_model": model or platform.machine()}


# windows per size bucket b (2^(b-1) < m <= 2^b) of the oracle's timing sample
_BUCKET_SAMPLE = {3: 400, 4: 400, 5: 300, 6: 200, 7: 100, 8: 40, 9: 16, 10: 8, 11: 4, 12: 3, 13: 2, 14: 1}


def oracle_bucket_cost(x, y, k=4, seed=9):
    """Seconds the oracle (one core) takes per window of each size bucket, on a seeded sample
    of windows of the pair (x, y)."""
    from oracle import oracle as O
    rng = np.random.default_rng(seed)
    n = len(x)
    cost = {}
    for b, cnt in _BUCKET_SAMPLE.items():
        lo, hi = max(k + 1, (1 << (b - 1)) + 1), 1 << b
        if lo > hi or hi > n:
            continue
        wins = []
        for _ in range(cnt):
            m = int(rng.integers(lo, hi + 1))
            st = int(rng.integers(0, n - m + 1))
            wins.append((st, m))
        t0 = time.perf_counter()
        for st, m in wins:
            O.ksg_window(x[st:st + m], y[st:st + m], k, points=False)
        cost[b] = (time.perf_counter() - t0) / cnt
    return cost


def config1_full():
    """Config 1 in full on the oracle: every window of 32, 64 and 128 points at stride 1 of the
    n = 2000 planted pair, and SYCOS_TD / SYCOS_BU with pruning off and on (sizes 32-256)."""
    from oracle import oracle as O
    from paper_2204_09131_gb300 import synth
    x, y = synth.planted_small_pair()
    wins = synth.stride_windows(len(x), [32, 64, 128])
    t0 = time.perf_counter()
    for st, m in wins:
        O.ksg_window(x[st:st + m], y[st:st + m], 4, points=False)
    t_sweep = time.perf_counter() - t0
    searches = {}
    for name, fn in (("td", O.search_td), ("bu", O.search_bu)):
        for pr in (0, 1):
            t0 = time.perf_counter()
            found, n_ev = fn(x, y, k=4, s_min=32, s_max=256, sigma=0.2, pruning=pr, seed=11)
            dt = time.perf_counter() - t0
            searches["%s_pruning%d" % (name, pr)] = {"evals": n_ev, "s": round(dt, 3),
                                                     "found": len(found)}
    return {"sweep_windows": len(wins), "sweep_s": round(t_sweep, 3),
            "sweep_evals_per_s": round(len(wins) / t_sweep, 1), "searches": searches}


def _oracle_search_job(job):
    """The oracle's SYCOS_TD + SYCOS_BU on the first `prefix` points of pair p (config-2
    shape); run in a spawned worker.  Returns the window scores it read."""
    p, length, prefix = job
    from oracle import oracle as O
    from paper_2204_09131_gb300 import synth
    x, y, _ = synth.planted_pair(2, p, length)
    _, n1 = O.search_td(x[:prefix], y[:prefix], **PARAMS)
    _, n2 = O.search_bu(x[:prefix], y[:prefix], **PARAMS)
    return n1 + n2


def oracle_multicore(n_pairs, length, prefix):
    """The same oracle searches on `n_pairs` pairs at once, one single-threaded process per
    core the host lets this process use (spawned workers, started before they are timed)."""
    import multiprocessing as mp
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    cores = max(1, min(cores, n_pairs))
    jobs = [(p, length, prefix) for p in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_job_ready, range(cores))   # workers up and imports done
        t0 = time.perf_counter()
        evals = sum(pool.map(_oracle_search_job, jobs, chunksize=1))
        secs = time.perf_counter() - t0
    return {"value": round(evals / secs, 2), "unit": "evals/s", "cores": cores, "evals": evals,
            "s": round(secs, 2),
            "sample": "SYCOS_TD + SYCOS_BU (pruning on, k=4, sizes 32-4096) on the first %d points "
                      "of pairs 0..%d, one process per core, all at once" % (prefix, cores - 1)}


def _oracle_job_ready(_):
    from oracle import oracle as O   # noqa: F401  (loads the oracle library in the worker)
    from paper_2204_09131_gb300 import synth   # noqa: F401
    return True


def cpu_baseline(pairs, decided_by_size=None, steps=1, prefix=12000, length=100000):
    """The oracle, single thread, on bounded samples of the workload.

    value: the step's decided windows divided by the oracle's extrapolated time for them --
    per size bucket, the oracle's mean seconds per window on a seeded sample of the pair's
    windows, times the step's decided windows in that bucket (labelled "extrapolated").
    Beside it: the oracle's SYCOS_TD + SYCOS_BU measured on the first `prefix` points of pair
    0 (real searches, also compared with the GPU's), and config 1 timed in full."""
    from oracle import oracle as O
    x, y = pairs[0]
    out = {"unit": "evals/s", "cores": 1, "kind": "oracle", "host": host_info()}
    cost = oracle_bucket_cost(x, y)
    out["per_bucket_s"] = {b: round(c, 7) for b, c in cost.items()}
    kw = dict(PARAMS)
    t0 = time.perf_counter()
    td, n1 = O.search_td(x[:prefix], y[:prefix], **kw)
    bu, n2 = O.search_bu(x[:prefix], y[:prefix], **kw)
    secs = time.perf_counter() - t0
    out["measured_search"] = {"value": round((n1 + n2) / secs, 2), "evals": n1 + n2, "s": round(secs, 2),
                              "sample": "SYCOS_TD + SYCOS_BU (pruning on, k=4, sizes 32-4096) on the "
                                        "first %d points of pair 0" % prefix}
    out["_searches"] = (td, bu)
    if decided_by_size is not None:
        per_step = [v / steps for v in decided_by_size]
        missing = [b for b, v in enumerate(per_step) if v > 0 and b not in cost]
        t_step = sum(v * cost.get(b, 0.0) for b, v in enumerate(per_step))
        out["value"] = round(sum(per_step) / t_step, 2) if t_step > 0 else None
        out["extrapolated"] = True
        out["extrapolated_s_per_step"] = round(t_step, 1)
        out["sample"] = ("extrapolated: the oracle's seconds per window by size bucket (seeded sample "
                         "of %d windows of pair 0, sizes 5-16384) x the step's decided windows per "
                         "bucket" % sum(_BUCKET_SAMPLE.values()))
        if missing:
            out["buckets_without_sample"] = missing
    else:
        out["value"] = out["measured_search"]["value"]
        out["sample"] = "oracle " + out["measured_search"]["sample"]
    out["config1_full"] = config1_full()
    out["multicore"] = oracle_multicore(len(pairs), length, prefix)
    return out


def reference_arm(args):
    """The oracle as it stands, on the host's cores: each step runs its SYCOS_TD + SYCOS_BU on
    the first 12,000 points of pairs 0 .. C-1 at once, one single-threaded process per usable
    core (C of them, spawned and warmed up before the clock starts)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import multiprocessing as mp
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    cores = max(1, min(cores, 16))
    prefix = 12000
    jobs = [(p, args.length, prefix) for p in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_job_ready, range(cores))

        def one_step():
            t0 = time.perf_counter()
            evals = sum(pool.map(_oracle_search_job, jobs, chunksize=1))
            dt = time.perf_counter() - t0
            return {"value": round(evals / dt, 2), "unit": "evals/s", "cores": cores, "kind": "oracle",
                    "host": host_info(),
                    "sample": "oracle SYCOS_TD + SYCOS_BU (pruning on, k=4, sizes 32-4096) on the first "
                              "%d points of pairs 0..%d, one process per core at once: %d window scores "
                              "in %.1f s" % (prefix, cores - 1, evals, dt)}

        for _ in range(args.warmup):   # untimed, like the other arm's warm-up steps
            one_step()
        vals = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            vals.append(one_step())
        ms = (time.perf_counter() - t0) * 1e3 / max(1, args.steps)
    v = statistics.median([c["value"] for c in vals])
    line = {"metric": METRIC, "value": v, "unit": "evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "isycos-td-bu-64x100k", "pairs": cores, "length": prefix,
                       "k": 4, "s_min": 32, "s_max": 4096, "pruning": 1},
            "cpu_baseline": dict(vals[-1], value=v),
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def case_windows(name, ids, length, rng):
    """Window lists of one MI batch shaped like the searches' frontiers."""
    starts, sizes, xs, ys = [], [], [], []

    def grid(m):
        d = max(5, m // 4)
        for a, b in ids:
            for t in range(0, length - m + 1, d):
                xs.append(a); ys.append(b); starts.append(t); sizes.append(m)

    if name.startswith("td") and name[2:].isdigit():
        grid(int(name[2:]))
    elif name == "mix":
        m = 4096
        while m >= 32:
            grid(m)
            m //= 2
    elif name == "chain":
        for a, b in ids:
            for t in range(0, 200 * 16, 16):
                xs.append(a); ys.append(b); starts.append(t); sizes.append(2048)
    elif name == "small":
        for a, b in ids:
            for _ in range(4000):
                m = int(np.exp(rng.uniform(np.log(32), np.log(128))))
                t = int(rng.integers(0, length - m))
                xs.append(a); ys.append(b); starts.append(t); sizes.append(m)
    elif name == "ring":
        for a, b in ids:
            for _ in range(2000):
                m = int(np.exp(rng.uniform(np.log(32), np.log(1024))))
                t = int(rng.integers(0, length - m))
                xs.append(a); ys.append(b); starts.append(t); sizes.append(m)
    else:
        raise SystemExit("unknown kernel case %r" % name)
    from paper_2204_09131_gb300 import api
    w = np.zeros(len(starts), dtype=api.WINDOW_DTYPE)
    w["xs"], w["ys"], w["start"], w["m"] = xs, ys, starts, sizes
    return w


def kernel_case(args):
    """One persistent MI launch on a fixed window list, timed by the library's CUDA events."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2204_09131_gb300 import api
    pairs = make_pairs(0, args.case_pairs, args.length)
    ctx = api.isycos_create(0, 0)
    ids = [(api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)) for x, y in pairs]
    api.isycos_set_option(ctx, api.OPT_KERNEL, args.kernel_opt)
    w = case_windows(args.kernel_case, ids, args.length, np.random.default_rng(5))
    for _ in range(args.warmup):
        api.isycos_mi_windows(ctx, w, 4)
    api.isycos_reset_stats(ctx)
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            api.isycos_mi_windows(ctx, w, 4)
    st = api.isycos_get_stats(ctx)
    ms = st["mi_kernel_ms"] / args.steps
    pairs_per_launch = st["pairs"] / args.steps
    clocks = clk.summary()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    f = clocks["sm_mhz"] or 2070.0
    peak = n_sm * 4 * 32 * f * 1e6
    ach = method_ops(st) / args.steps / (ms / 1e3)
    bfe = OPS_PER_PAIR * pairs_per_launch / (ms / 1e3)
    line = {"kernel_case": args.kernel_case, "kernel_opt": args.kernel_opt, "windows": int(len(w)),
            "ms_per_launch": round(ms, 4),
            "evals_per_s": round(len(w) / (ms / 1e3), 1),
            "pairs_per_s": round(pairs_per_launch / (ms / 1e3), 1),
            "roofline": {"bound": "alu", "achieved": round(ach / 1e9, 1), "peak": round(peak / 1e9, 1),
                         "unit": "Glane-op/s", "frac": round(ach / peak, 4),
                         "work_per_launch": {f: int(st[f] / args.steps) for f in OPS_PER_UNIT},
                         "brute_force_equivalent_frac": round(bfe / peak, 4)},
            "clocks": clocks}
    if args.kernel_case == "chain":
        # the same windows through the incremental kernel, one chain per pair
        t_inc = 0.0
        api.isycos_reset_stats(ctx)
        for _ in range(args.steps):
            t0 = time.perf_counter()
            for a, b in ids:
                sel = (w["xs"] == a)
                api.isycos_mi_chain(ctx, a, b, w["start"][sel], w["m"][sel], 4)
            t_inc += time.perf_counter() - t0
        st2 = api.isycos_get_stats(ctx)
        line["incremental"] = {"s_per_pass": round(t_inc / args.steps, 4),
                               "full_points_frac": round(st2["incr_full_points"] / max(1, int(w["m"].sum()) * args.steps), 4)}
    if args.plain:
        sub = w[: max(1, min(len(w), 2000))]
        t0 = time.perf_counter()
        api.isycos_mi_windows_plain(ctx, sub, 4)
        t_plain = time.perf_counter() - t0
        t0 = time.perf_counter()
        api.isycos_mi_windows(ctx, sub, 4)
        t_batch = time.perf_counter() - t0
        line["plain_vs_batched"] = {"windows": int(len(sub)), "plain_s": round(t_plain, 4),
                                    "batched_s": round(t_batch, 4)}
    print(json.dumps(line), flush=True)
    api.isycos_destroy(ctx)


def search_case(args):
    """Searches of one kind over a few pairs: time per pass and the library's per-size
    launch statistics (windows, launches and summed launch time by window-size bucket)."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2204_09131_gb300 import api
    pairs = make_pairs(0, args.case_pairs, args.length)
    ctx = api.isycos_create(0, 0)
    if args.lanes:
        api.isycos_set_option(ctx, api.OPT_LANES, args.lanes)
    if args.speculation >= 0:
        api.isycos_set_option(ctx, api.OPT_SPECULATION, args.speculation)
    ids = [(api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)) for x, y in pairs]
    # the MI path per window size, chosen on this GPU as in the default step
    tune = api.isycos_autotune(ctx, PARAMS["k"])
    extra = {"td": [dict(mode=0)], "bu": [dict(mode=1)], "mix": [dict(mode=0), dict(mode=1)],
             "select": [dict(mode=2)], "chunked": [dict(mode=1, chunks=8)]}[args.search_case]
    qs = [(a, b, 0, args.length, dict(PARAMS, **e)) for e in extra for a, b in ids]
    for _ in range(args.warmup):
        api.isycos_search_queries(ctx, qs)
    torch.cuda.synchronize()
    api.isycos_reset_stats(ctx)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        api.isycos_search_queries(ctx, qs)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.steps
    st = api.isycos_get_stats(ctx)
    k = args.steps
    line = {"search_case": args.search_case, "pairs": args.case_pairs, "length": args.length,
            "lanes": args.lanes, "speculation": args.speculation,
            "sorted_buckets": tune["sorted_buckets"],
            "s_per_pass": round(dt, 4), "decided_windows": st["decided_windows"] // k,
            "gpu_windows": st["windows"] // k, "launches": st["launches"] // k,
            "kernel_ms": round(st["mi_kernel_ms"] / k, 2),
            "windows_by_size": [v // k for v in st["windows_by_size"]],
            "launches_by_size": [v // k for v in st["launches_by_size"]],
            "launch_ms_by_size": [round(v / k, 2) for v in st["launch_ms_by_size"]],
            "decided_by_size": [v // k for v in st["decided_by_size"]],
            "dev_queries": st["dev_queries"] // k, "dev_rounds": st["dev_rounds"] // k,
            "dev_cycles": [v // k for v in st["dev_cycles"]],
            "work": {f: st[f] // k for f in ("work_bf", "work_scan", "work_search", "work_sort")}}
    print(json.dumps(line), flush=True)
    api.isycos_destroy(ctx)


def serving_case(args):
    """Continuous batching at scale, swept over load: --serve-series resident series of
    --serve-length points, capacity measured with --serve-calibrate queries submitted at once,
    then Poisson streams of --serve-queries queries at the fractions --serve-rates of it."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2204_09131_gb300 import api
    ctx = api.isycos_create(0, 0)
    n_pairs, length = max(1, args.serve_series // 2), args.serve_length
    ids = put_serving_series(api, ctx, n_pairs, length)
    api.isycos_autotune(ctx, PARAMS["k"])
    cal_q = serving_queries(ids, length, args.serve_calibrate, 1)
    _, _, wall = serve_stream(api, ctx, cal_q, [0.0] * len(cal_q))
    capacity = len(cal_q) / wall
    sweep = []
    for f in [float(v) for v in args.serve_rates.split(",")]:
        qs = serving_queries(ids, length, args.serve_queries, 100 + int(f * 100))
        gaps = np.random.default_rng(7).exponential(1.0 / (f * capacity), len(qs))
        lat, wait, wall = serve_stream(api, ctx, qs, gaps)
        sweep.append({"rate_fraction": f, "arrival_qps": round(f * capacity, 2), "queries": len(qs),
                      "p50_ms": round(float(np.percentile(lat, 50)), 2),
                      "p99_ms": round(float(np.percentile(lat, 99)), 2),
                      "throughput_qps": round(len(qs) / wall, 2),
                      "admission_wait_p99_ms": round(float(np.percentile(wait, 99)), 3)})
    st = api.isycos_get_stats(ctx)
    print(json.dumps({"serving_case": True, "series": 2 * n_pairs, "length": length,
                      "capacity_qps": round(capacity, 2), "sweep": sweep,
                      "queries_done": st["queries_done"]}), flush=True)
    api.isycos_destroy(ctx)


def main():
    args = parse()
    if args.serving_case:
        return serving_case(args)
    if args.search_case:
        return search_case(args)
    if args.impl == "reference":
        return reference_arm(args)
    if args.kernel_case:
        return kernel_case(args)
    if args.stress_case:
        import torch
        torch.cuda.set_device(0)
        import __graft_entry__
        __graft_entry__.build()
        print(json.dumps(pruning_stress(args)), flush=True)
        return
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_2204_09131_gb300 import api

    pairs = make_pairs(rank, args.pairs, args.length, world)
    ctx = api.isycos_create(local, 0)
    ids = [(api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)) for x, y in pairs]
    l2buf = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    # per-bucket choice between the brute-force and sorted MI paths, timed on this GPU
    tune = api.isycos_autotune(ctx, PARAMS["k"])

    for _ in range(args.warmup):
        run_step(api, ctx, ids, args.length)
    torch.cuda.synchronize()

    api.isycos_reset_stats(ctx)
    times = []
    found = 0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush_l2(torch, l2buf)
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            found = run_step(api, ctx, ids, args.length)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    st = api.isycos_get_stats(ctx)
    total_ms = sum(times)
    # value: window MIs that the searches' decisions read (the sequential algorithms' count,
    # the unit of the oracle baseline); windows evaluated on the GPU including speculative
    # ones are reported beside it
    windows = st["decided_windows"]
    gpu_windows = st["windows"]
    pairs_cnt = st["pairs"]
    if world > 1:
        t = torch.tensor([total_ms, windows, pairs_cnt], dtype=torch.float64, device="cuda")
        mx = t.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        total_ms_max = mx[0].item()
        windows_all, pairs_all = t[1].item(), t[2].item()
    else:
        total_ms_max, windows_all, pairs_all = total_ms, windows, pairs_cnt
    value = windows_all / (total_ms_max / 1e3)
    pairs_per_s = pairs_all / (total_ms_max / 1e3)

    # e2e: series uploaded from pinned host memory, searches, results read back; repeated
    # min(steps, 5) times (each an upload, a step and the drops), after one untimed repetition
    e2e = None
    if rank == 0:
        pinned = [(torch.from_numpy(x).pin_memory(), torch.from_numpy(y).pin_memory()) for x, y in pairs]
        host = [t.numpy() for xy in pinned for t in xy]

        def e2e_step():
            flat = api.isycos_put_series_many(ctx, host)
            eids = list(zip(flat[0::2], flat[1::2]))
            st0 = api.isycos_get_stats(ctx)
            nf = run_step(api, ctx, eids, args.length)
            st1 = api.isycos_get_stats(ctx)
            for a, b in eids:
                api.isycos_drop_series(ctx, a)
                api.isycos_drop_series(ctx, b)
            return st1["decided_windows"] - st0["decided_windows"], nf

        e2e_step()
        torch.cuda.synchronize()
        reps = max(1, min(args.steps, 5))
        n_dec, nfound = 0, 0
        t0 = time.perf_counter()
        for _ in range(reps):
            d, nfound = e2e_step()
            n_dec += d
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": round(n_dec / dt, 2), "unit": "evals/s",
               "h2d_bytes_per_step": int(2 * len(pairs) * args.length * 4),
               "d2h_bytes_per_step": int(nfound * 32), "steps": reps}

    # roofline of the dominant kernel (the batched MI kernel): algorithmic lane operations
    # per launch over its event-timed duration, against the CUDA-core issue peak
    clocks = clk.summary()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    f_mhz = clocks["sm_mhz"] or 2070.0
    peak = n_sm * 4 * 32 * f_mhz * 1e6 / 1e9        # G lane-ops / s
    kms = st["mi_kernel_ms"]
    ops = method_ops(st)
    achieved = ops / (kms / 1e3) / 1e9 if kms > 0 else None
    bfe = (OPS_PER_PAIR * pairs_cnt) / (kms / 1e3) / 1e9 if kms > 0 else None
    roof = {"bound": "alu", "achieved": round(achieved, 1) if achieved else None,
            "peak": round(peak, 1), "unit": "Glane-op/s",
            "frac": round(achieved / peak, 4) if achieved else None, "traffic": None,
            "kernel": "ksg_batched_kernel", "kernel_ms_per_step": round(kms / args.steps, 3),
            "kernel_share_of_step": round(kms / total_ms, 4) if total_ms else None,
            "peak_basis": "%d SMs x 4 warp-instr/clk x 32 lanes x %.0f MHz (median SM clock "
                          "sampled during the timed region)" % (n_sm, f_mhz),
            "work_basis": "the work the kernels did, counted per launch: brute-force point x "
                          "candidate evaluations x 11, sorted-path outward-scan visits x 6, "
                          "binary-search steps x 5, bitonic compare-exchanges x 4 lane-ops, "
                          "over the union of the batched kernel's launch intervals",
            "work_per_step": {f: int(st[f] / args.steps) for f in OPS_PER_UNIT},
            "brute_force_equivalent": {"achieved": round(bfe, 1) if bfe else None,
                                       "frac": round(bfe / peak, 4) if bfe else None,
                                       "basis": "11 lane-ops per ordered pair m(m-1) of every "
                                                "evaluated window, as if all ran by brute force"}}

    serving = None
    if rank == 0 and not args.no_serving:
        serving = serving_config4(args)
    stress = None
    if rank == 0 and not args.no_stress:
        stress = pruning_stress(args)

    # the plain form (one window per launch) against the batched form, on 2,000 windows shaped
    # like the BU rings of the step (32-1024 points)
    plain = None
    if rank == 0:
        wr = case_windows("ring", ids[:1], args.length, np.random.default_rng(5))
        api.isycos_mi_windows(ctx, wr, PARAMS["k"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rp = api.isycos_mi_windows_plain(ctx, wr, PARAMS["k"])
        t_plain = time.perf_counter() - t0
        t0 = time.perf_counter()
        rb = api.isycos_mi_windows(ctx, wr, PARAMS["k"])
        t_batch = time.perf_counter() - t0
        diff = np.nonzero(rp["s_psi"] != rb["s_psi"])[0]
        plain = {"windows": int(len(wr)), "plain_evals_per_s": round(len(wr) / t_plain, 1),
                 "batched_evals_per_s": round(len(wr) / t_batch, 1),
                 "speedup": round(t_plain / t_batch, 1),
                 "same_results": bool(diff.size == 0)}
        if diff.size:
            plain["differing"] = {"count": int(diff.size), "sizes": [int(v) for v in wr["m"][diff[:8]]]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(pairs, st["decided_by_size"], args.steps, length=args.length)
        # the GPU's searches on the same prefix must return the oracle's windows
        td, bu = cpu.pop("_searches")
        got = api.isycos_search_queries(ctx, [(ids[0][0], ids[0][1], 0, 12000, dict(PARAMS, mode=0)),
                                              (ids[0][0], ids[0][1], 0, 12000, dict(PARAMS, mode=1))])
        same = all([(int(a), int(b)) for a, b in zip(g["t_s"], g["t_e"])] == [(a, b) for a, b, _, _ in r]
                   for g, r in ((got[0], td), (got[1], bu)))
        cpu["measured_search"]["gpu_same_windows"] = bool(same)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms_max / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "isycos-td-bu-64x100k", "pairs_per_gpu": args.pairs,
                       "length": args.length, "k": 4, "s_min": 32, "s_max": 4096,
                       "sigma": 0.2, "pruning": 1,
                       "searches": "SYCOS_TD and SYCOS_BU queries of every pair, concurrently",
                       "l2": "flushed between timed steps (256 MiB write)",
                       "autotune": {"sorted_buckets": tune["sorted_buckets"],
                                    "sort_min": tune["sort_min"], "nt_switch": tune["nt_switch"],
                                    "window_size": tune["window_size"],
                                    "brute_ms": tune["brute_ms"], "sorted_ms": tune["sorted_ms"],
                                    "crossover": tune["crossover"], "nt_ms": tune["nt_ms"]}},
            "pairs_per_s": round(pairs_per_s, 1),
            "pairs_note": "brute-force-equivalent ordered pairs m(m-1) per evaluated window",
            "windows_per_step": int(windows_all / args.steps),
            "gpu_windows_per_step": int(gpu_windows / args.steps),
            "gpu_windows_per_s": round(gpu_windows / (total_ms / 1e3), 1),
            "found_windows_per_step": found,
            "incremental_windows_per_step": int(st["incr_windows"] / args.steps),
            "gpu_launches": int(st["launches"]),
            "roofline": roof, "clocks": clocks, "e2e": e2e, "serving": serving,
            "plain_vs_batched": plain, "pruning_stress": stress,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    api.isycos_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
