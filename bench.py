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


def serving_probe(api, ctx, ids, length, n_queries=200, rate_hz=None):
    """Poisson stream of search queries over the resident pairs (reduced size)."""
    rng = np.random.default_rng(4)
    queries = []
    for i in range(n_queries):
        a, b = ids[int(rng.integers(0, len(ids)))]
        span = int(np.exp(rng.uniform(np.log(1000), np.log(length))))
        lo = int(rng.integers(0, length - span + 1))
        s_max = int(2 ** rng.integers(8, 13))
        s_max = max(64, min(s_max, span // 2))
        queries.append((a, b, lo, lo + span, dict(PARAMS, s_max=s_max, mode=int(i % 2))))
    # calibrate: one query's service time
    t0 = time.perf_counter()
    api.isycos_search(ctx, *queries[0][:4], queries[0][4])
    t1 = time.perf_counter() - t0
    rate = rate_hz or max(1.0, 0.7 * 32 / max(t1, 1e-4))
    gaps = rng.exponential(1.0 / rate, n_queries)
    tickets = []
    start = time.perf_counter()
    nxt = start
    done = {}
    for q, g in zip(queries, gaps):
        nxt += g
        while time.perf_counter() < nxt:
            for t in tickets:
                if t not in done:
                    r = api.isycos_serve_poll(ctx, t)
                    if r is not None:
                        done[t] = r[1]
            time.sleep(0.0005)
        tickets.append(api.isycos_serve_submit(ctx, *q[:4], q[4]))
    while len(done) < len(tickets):
        for t in tickets:
            if t not in done:
                r = api.isycos_serve_poll(ctx, t)
                if r is not None:
                    done[t] = r[1]
        time.sleep(0.0005)
    wall = time.perf_counter() - start
    lat = np.array([done[t] for t in tickets])
    return {"queries": n_queries, "arrival_rate_hz": round(rate, 2),
            "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "throughput_qps": round(n_queries / wall, 2)}


def cpu_baseline(pairs, budget_s=15.0):
    """The oracle, single thread, on a bounded sample: TD then BU (pruning on) on prefixes of
    pair 0 until the CPU budget is spent; evals/s = windows scored / seconds."""
    from oracle import oracle as O
    x, y = pairs[0]
    kw = dict(PARAMS)
    evals, secs = 0, 0.0
    span = 12000
    t0 = time.perf_counter()
    _, n1 = O.search_td(x[:span], y[:span], **kw)
    _, n2 = O.search_bu(x[:span], y[:span], **kw)
    secs = time.perf_counter() - t0
    evals = n1 + n2
    return {"value": round(evals / secs, 2), "unit": "evals/s", "cores": 1, "kind": "oracle",
            "sample": "oracle SYCOS_TD + SYCOS_BU (pruning on, k=4, sizes 32-4096) on the first "
                      "%d points of pair 0: %d window scores in %.1f s" % (span, evals, secs)}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    pairs = make_pairs(0, 1, args.length)
    for _ in range(args.warmup):   # untimed, like the other arm's warm-up steps
        cpu_baseline(pairs)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(pairs))
    ms = (time.perf_counter() - t0) * 1e3 / max(1, args.steps)
    v = statistics.median([c["value"] for c in vals])
    line = {"metric": METRIC, "value": v, "unit": "evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "isycos-td-bu-64x100k", "pairs": 1, "length": 12000,
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
    """Continuous batching at scale: random queries (random pair of the resident series, range
    log-uniform in [1e3, length], s_max a power of two log-uniform in [256, 16384] clipped to
    range / 2, SYCOS_TD and SYCOS_BU alternating) submitted as Poisson streams at fractions
    of the capacity measured with the same kind of queries submitted all at once."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2204_09131_gb300 import api, synth
    ctx = api.isycos_create(0, 0)
    n_pairs = max(1, args.serve_series // 2)
    ids = []
    for p in range(n_pairs):
        x, y, _ = synth.planted_pair(4, p, args.serve_length)
        ids.append((api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)))
    api.isycos_autotune(ctx, PARAMS["k"])
    length = args.serve_length

    def make_queries(n, seed):
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

    def run(qs, gaps):
        tickets, done = [], {}
        start = time.perf_counter()
        nxt = start
        for q, g in zip(qs, gaps):
            nxt += g
            while time.perf_counter() < nxt:
                time.sleep(0.0002)
            tickets.append(api.isycos_serve_submit(ctx, *q[:4], q[4]))
            for t in tickets[-64:]:
                if t not in done:
                    r = api.isycos_serve_poll(ctx, t)
                    if r is not None:
                        done[t] = r[1]
        while len(done) < len(tickets):
            for t in tickets:
                if t not in done:
                    r = api.isycos_serve_poll(ctx, t)
                    if r is not None:
                        done[t] = r[1]
            time.sleep(0.001)
        wall = time.perf_counter() - start
        lat = np.array([done[t] for t in tickets])
        return {"queries": len(qs), "p50_ms": round(float(np.percentile(lat, 50)), 2),
                "p99_ms": round(float(np.percentile(lat, 99)), 2),
                "throughput_qps": round(len(qs) / wall, 2)}

    cal = run(make_queries(min(256, args.serve_queries), 1), [0.0] * min(256, args.serve_queries))
    capacity = cal["throughput_qps"]
    sweep = []
    for f in [float(v) for v in args.serve_rates.split(",")]:
        qs = make_queries(args.serve_queries, 100 + int(f * 100))
        gaps = np.random.default_rng(7).exponential(1.0 / (f * capacity), len(qs))
        r = run(qs, gaps)
        r["rate_fraction"] = f
        r["arrival_qps"] = round(f * capacity, 2)
        sweep.append(r)
    st = api.isycos_get_stats(ctx)
    line = {"serving_case": True, "series": 2 * n_pairs, "length": length,
            "capacity_qps": capacity, "calibration": cal, "sweep": sweep,
            "queries_done": st["queries_done"]}
    print(json.dumps(line), flush=True)
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

    # e2e: series uploaded from pinned host memory, searches, results read back.
    e2e = None
    if rank == 0:
        pinned = [(torch.from_numpy(x).pin_memory(), torch.from_numpy(y).pin_memory()) for x, y in pairs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eids = []
        for x, y in pinned:
            eids.append((api.isycos_put_series(ctx, x.numpy()), api.isycos_put_series(ctx, y.numpy())))
        st0 = api.isycos_get_stats(ctx)
        nfound = run_step(api, ctx, eids, args.length)
        st1 = api.isycos_get_stats(ctx)
        st0["windows"], st1["windows"] = st0["decided_windows"], st1["decided_windows"]
        for a, b in eids:
            api.isycos_drop_series(ctx, a)
            api.isycos_drop_series(ctx, b)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": round((st1["windows"] - st0["windows"]) / dt, 2), "unit": "evals/s",
               "h2d_bytes_per_step": int(2 * len(pairs) * args.length * 4),
               "d2h_bytes_per_step": int(nfound * 32)}

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
        serving = serving_probe(api, ctx, ids, args.length)

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
        cpu = cpu_baseline(pairs)

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
                                    "window_size": tune["window_size"],
                                    "brute_ms": tune["brute_ms"], "sorted_ms": tune["sorted_ms"]}},
            "pairs_per_s": round(pairs_per_s, 1),
            "pairs_note": "brute-force-equivalent ordered pairs m(m-1) per evaluated window",
            "windows_per_step": int(windows_all / args.steps),
            "gpu_windows_per_step": int(gpu_windows / args.steps),
            "gpu_windows_per_s": round(gpu_windows / (total_ms / 1e3), 1),
            "found_windows_per_step": found,
            "incremental_windows_per_step": int(st["incr_windows"] / args.steps),
            "gpu_launches": int(st["launches"]),
            "roofline": roof, "clocks": clocks, "e2e": e2e, "serving": serving,
            "plain_vs_batched": plain,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    api.isycos_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
