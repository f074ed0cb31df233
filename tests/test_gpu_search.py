"""Search and serving on the GPU against the oracle's sequential searches (GPU).

isycos_search batches window scores (a whole TD layer grid, a whole BU ring) and replays the
sequential decisions; the selected windows must equal the oracle's Algorithm 1 / Algorithm 2
(with and without the Sec. 6 pruning) exactly, and the scores of the selected windows within
1e-12.
"""
import threading
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2204_09131_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2204_09131_gb300 import api
    assert torch.cuda.is_available()
    c = api.Context(0)
    yield c.h
    c.close()


def _api():
    from paper_2204_09131_gb300 import api
    return api


def _same(got, ref):
    g = [(int(a), int(b)) for a, b in zip(got["t_s"], got["t_e"])]
    r = [(a, b) for a, b, _, _ in ref]
    assert g == r, (g, r)
    for (a, b, sc, mi), gs, gm in zip(ref, got["score"], got["mi"]):
        assert abs(gs - sc) <= 1e-12 and abs(gm - mi) <= 1e-12


PARAMS = [
    dict(mode=0, pruning=0), dict(mode=0, pruning=1),
    dict(mode=1, pruning=0), dict(mode=1, pruning=1),
    dict(mode=0, pruning=1, score_kind=1, sigma=0.5, tau=0.1),
    dict(mode=1, pruning=1, score_kind=1, sigma=0.5, tau=0.1, seed=5),
    dict(mode=0, delta_td=24, s_min=40, s_max=200),          # delta does not divide s_w
    dict(mode=1, delta_bu=5, h=3, t_max_idle=1, seed=77),
]


@pytest.mark.parametrize("extra", PARAMS, ids=lambda d: ",".join("%s=%s" % kv for kv in d.items()))
def test_search_matches_oracle_planted_pair(ctx, extra):
    api = _api()
    x, y = synth.planted_small_pair()
    kw = dict(k=4, s_min=32, s_max=256, sigma=0.2, seed=11)
    kw.update(extra)
    xs = api.isycos_put_series(ctx, x)
    ys = api.isycos_put_series(ctx, y)
    got = api.isycos_search(ctx, xs, ys, 0, len(x), kw)
    okw = dict(kw)
    mode = okw.pop("mode")
    ref, _ = (O.search_td if mode == 0 else O.search_bu)(x, y, **okw)
    _same(got, ref)
    api.isycos_drop_series(ctx, xs)
    api.isycos_drop_series(ctx, ys)


@pytest.mark.parametrize("mode", [0, 1])
def test_search_subrange_and_quantised(ctx, mode):
    api = _api()
    x, y, _ = synth.planted_pair(2, 3, 12000, len_lo=50, len_hi=1500)
    x, y = synth.quantize(x), synth.quantize(y)
    xs = api.isycos_put_series(ctx, x)
    ys = api.isycos_put_series(ctx, y)
    kw = dict(k=3, s_min=32, s_max=512, sigma=0.15, pruning=1, seed=2)
    got = api.isycos_search(ctx, xs, ys, 1000, 9000, dict(kw, mode=mode))
    ref, _ = (O.search_td if mode == 0 else O.search_bu)(x, y, t_begin=1000, t_end=9000, **kw)
    _same(got, ref)


def test_search_many_equals_single_searches(ctx):
    api = _api()
    ids = []
    for p in range(4):
        x, y, _ = synth.planted_pair(2, p, 8000, len_lo=50, len_hi=1000)
        ids.append((api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)))
    for mode in (0, 1):
        prm = dict(k=4, s_min=32, s_max=512, mode=mode, pruning=1, seed=4)
        many = api.isycos_search_many(ctx, [a for a, _ in ids], [b for _, b in ids], [0] * 4,
                                      [8000] * 4, prm)
        for (a, b), got in zip(ids, many):
            one = api.isycos_search(ctx, a, b, 0, 8000, prm)
            assert np.array_equal(one, got)


def test_search_rejects_bad_params(ctx):
    api = _api()
    x = synth.normal(3, 500).astype(np.float32)
    xs = api.isycos_put_series(ctx, x)
    for bad in (dict(s_min=4, k=4), dict(s_min=64, s_max=32), dict(s_max=20000), dict(mode=3),
                dict(k=9, s_min=32)):
        with pytest.raises(api.IsycosError) as e:
            api.isycos_search(ctx, xs, xs, 0, 500, bad)
        assert e.value.status == api.E_INVAL
    with pytest.raises(api.IsycosError):
        api.isycos_search(ctx, xs, xs, 0, 501, {})
    with pytest.raises(api.IsycosError) as e:
        api.isycos_search(ctx, xs, 12345, 0, 100, {})
    assert e.value.status == api.E_NOTFOUND


def test_search_truncation_reports_needed(ctx):
    import ctypes
    api = _api()
    x, y = synth.planted_small_pair()
    xs = api.isycos_put_series(ctx, x)
    ys = api.isycos_put_series(ctx, y)
    full = api.isycos_search(ctx, xs, ys, 0, 2000, dict(k=4, s_min=32, s_max=256))
    assert len(full) >= 2
    out = np.empty(1, dtype=api.RESULT_DTYPE)
    n = ctypes.c_int64()
    p = api.isycos_params_default(k=4, s_min=32, s_max=256)
    st = api.lib().isycos_search(ctx, xs, ys, 0, 2000, ctypes.byref(p), out.ctypes.data, 1,
                                 ctypes.byref(n))
    assert st == api.E_TRUNC and n.value == len(full)


def _serve_all(ctx, queries, params):
    api = _api()
    tickets = [api.isycos_serve_submit(ctx, *q, params) for q in queries]
    res = {}
    deadline = time.time() + 300
    while len(res) < len(tickets) and time.time() < deadline:
        for t in tickets:
            if t in res:
                continue
            r = api.isycos_serve_poll(ctx, t)
            if r is not None:
                res[t] = r
        time.sleep(0.002)
    assert len(res) == len(tickets)
    return [res[t] for t in tickets]


def test_serving_same_alone_and_in_the_mix(ctx):
    api = _api()
    pairs = []
    for p in range(6):
        x, y, _ = synth.planted_pair(4, p, 10000, len_lo=50, len_hi=2000)
        pairs.append((api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)))
    queries = []
    rng = np.random.default_rng(1)
    for i in range(24):
        a, b = pairs[i % 6]
        lo = int(rng.integers(0, 5000))
        hi = int(rng.integers(lo + 600, 10000))
        queries.append((a, b, lo, hi))
    for mode in (0, 1):
        prm = dict(k=4, s_min=32, s_max=512, mode=mode, pruning=1, seed=9)
        mixed = _serve_all(ctx, queries, prm)
        for q, (wins, lat) in zip(queries, mixed):
            alone = api.isycos_search(ctx, *q, prm)
            assert np.array_equal(alone, wins)
            assert lat > 0
    s = api.isycos_get_stats(ctx)
    assert s["queries_done"] >= 48


def test_serving_concurrent_submitters_and_cancel(ctx):
    api = _api()
    x, y, _ = synth.planted_pair(4, 9, 20000)
    a, b = api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)
    prm = dict(k=4, s_min=32, s_max=1024, mode=0)
    expect = api.isycos_search(ctx, a, b, 0, 20000, prm)
    out = {}

    def worker(i):
        t = api.isycos_serve_submit(ctx, a, b, 0, 20000, prm)
        while True:
            r = api.isycos_serve_poll(ctx, t)
            if r is not None:
                out[i] = r[0]
                return
            time.sleep(0.001)

    th = [threading.Thread(target=worker, args=(i,)) for i in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert len(out) == 4 and all(np.array_equal(v, expect) for v in out.values())
    # cancel a query: its poll reports E_CANCELED (whether it was queued or running)
    t = api.isycos_serve_submit(ctx, a, b, 0, 20000, dict(prm, mode=1))
    api.isycos_serve_cancel(ctx, t)
    deadline = time.time() + 60
    while time.time() < deadline:
        try:
            r = api.isycos_serve_poll(ctx, t)
        except api.IsycosError as e:
            assert e.status == api.E_CANCELED
            break
        if r is not None:      # finished before the cancel reached it
            break
        time.sleep(0.001)
    with pytest.raises(api.IsycosError) as e:
        api.isycos_serve_poll(ctx, 987654321)
    assert e.value.status == api.E_NOTFOUND


def test_serving_admission_under_a_small_budget():
    """A context whose budget leaves room for one query's work buffers at a time (each TD
    query here is estimated at 360 KB: 2,501 windows of the s_w = 32 layer, twice for buffer
    growth) still completes every query, one after another, with the same results."""
    api = _api()
    x, y, _ = synth.planted_pair(4, 11, 20000)
    c = api.Context(0, mem_budget_bytes=(2 * 20000 * 4) + 2 * 8 * 16386 + 500_000)
    try:
        a, b = api.isycos_put_series(c.h, x), api.isycos_put_series(c.h, y)
        prm = dict(k=4, s_min=32, s_max=256, mode=0)
        res = _serve_all(c.h, [(a, b, 0, 20000)] * 3, prm)
        ref = api.isycos_search(c.h, a, b, 0, 20000, prm)
        assert all(np.array_equal(r[0], ref) for r in res)
    finally:
        c.close()


@pytest.mark.parametrize("opt", [0, 1, 2])
@pytest.mark.parametrize("extra", [dict(mode=0, delta_td=4, s_min=48, s_max=192, pruning=1),
                                   dict(mode=1, pruning=1, seed=3),
                                   dict(mode=1, pruning=0, s_max=1024, seed=8)],
                         ids=["td-small-delta", "bu-pruning", "bu-large"])
def test_search_with_incremental_updates(ctx, opt, extra):
    """Searches whose frontiers run through the incremental kernel (opt 2: every chain;
    opt 1: chains the cost model picks; opt 0: none) give the oracle's windows."""
    api = _api()
    x, y = synth.planted_small_pair()
    kw = dict(k=4, s_min=32, s_max=256, sigma=0.2, seed=11)
    kw.update(extra)
    xs = api.isycos_put_series(ctx, x)
    ys = api.isycos_put_series(ctx, y)
    api.isycos_set_option(ctx, api.OPT_INCREMENTAL, opt)
    api.isycos_reset_stats(ctx)
    try:
        got = api.isycos_search(ctx, xs, ys, 0, len(x), kw)
    finally:
        api.isycos_set_option(ctx, api.OPT_INCREMENTAL, 1)
    st = api.isycos_get_stats(ctx)
    if opt == 2:
        assert st["incr_windows"] > 0
    if opt == 0:
        assert st["incr_windows"] == 0
    okw = dict(kw)
    mode = okw.pop("mode")
    ref, _ = (O.search_td if mode == 0 else O.search_bu)(x, y, **okw)
    _same(got, ref)


@pytest.mark.parametrize("mode", [0, 1])
def test_decided_windows_equal_the_oracles_evaluations(ctx, mode):
    """Batching evaluates extra (speculative) windows; the decisions read exactly the scores
    the sequential algorithm computes, so the decided-window count equals the oracle's."""
    api = _api()
    x, y = synth.planted_small_pair()
    kw = dict(k=4, s_min=32, s_max=256, sigma=0.2, pruning=1, seed=21)
    xs, ys = api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)
    api.isycos_reset_stats(ctx)
    api.isycos_search(ctx, xs, ys, 0, len(x), dict(kw, mode=mode))
    st = api.isycos_get_stats(ctx)
    _, n_evals = (O.search_td if mode == 0 else O.search_bu)(x, y, **kw)
    assert st["decided_windows"] == n_evals
    assert st["windows"] >= n_evals


def test_search_queries_mixed_modes_equal_single_searches(ctx):
    api = _api()
    ids = []
    for p in range(3):
        x, y, _ = synth.planted_pair(2, 10 + p, 6000, len_lo=50, len_hi=800)
        ids.append((api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)))
    queries = []
    for i, (a, b) in enumerate(ids):
        queries.append((a, b, 0, 6000, dict(k=4, s_min=32, s_max=512, mode=0, pruning=i % 2)))
        queries.append((a, b, 500, 5500, dict(k=3, s_min=40, s_max=300, mode=1, pruning=1, seed=i)))
    got = api.isycos_search_queries(ctx, queries)
    for q, g in zip(queries, got):
        assert np.array_equal(api.isycos_search(ctx, *q), g)


@pytest.mark.parametrize("case", ["planted", "weak"])
def test_selection_matches_oracle(ctx, case):
    """iSYCOS selection (Algorithm 3): the GPU search samples the same partitions, scores TD
    and BU with the same deterministic runtime, selects the same search and returns its
    windows; its decided-window count equals the oracle's."""
    api = _api()
    if case == "planted":
        x, y = synth.planted_small_pair()
    else:
        x, y, _ = synth.planted_pair(3, 1, 4000, coverage=0.1, len_lo=40, len_hi=200)
    kw = dict(k=4, s_min=32, s_max=256, sigma=0.2, pruning=1, seed=17)
    xs, ys = api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)
    api.isycos_reset_stats(ctx)
    got = api.isycos_search(ctx, xs, ys, 0, len(x), dict(kw, mode=2, sel_partitions=8,
                                                          sel_samples=3))
    st = api.isycos_get_stats(ctx)
    ref, n, sel, _ = O.search_auto(x, y, partitions=8, samples=3, **kw)
    _same(got, ref)
    assert st["decided_windows"] == n


@pytest.mark.parametrize("extra", [dict(mode=0, chunks=4), dict(mode=1, chunks=3, pruning=1),
                                   dict(mode=0, chunks=7, pruning=1, s_max=128),
                                   dict(mode=2, chunks=3, sel_partitions=8, sel_samples=3)],
                         ids=lambda d: ",".join("%s=%s" % kv for kv in d.items()))
def test_chunked_search_matches_oracle(ctx, extra):
    """Algorithm 4: the range is searched as overlapping chunks; the GPU's chunk searches run
    batched together and must return the oracle's concatenated, t_s-sorted windows and its
    evaluation count."""
    api = _api()
    x, y = synth.planted_small_pair()
    kw = dict(k=4, s_min=32, s_max=256, sigma=0.2, seed=9)
    kw.update(extra)
    xs, ys = api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)
    api.isycos_reset_stats(ctx)
    got = api.isycos_search(ctx, xs, ys, 0, len(x), kw)
    st = api.isycos_get_stats(ctx)
    okw = dict(kw)
    mode = okw.pop("mode")
    if mode == 2:
        ref, n, _, _ = O.search_auto(x, y, partitions=okw.pop("sel_partitions"),
                                     samples=okw.pop("sel_samples"), **okw)
    else:
        ref, n = O.search_chunked(x, y, mode=mode, **okw)
    _same(got, ref)
    assert st["decided_windows"] == n
    api.isycos_drop_series(ctx, xs)
    api.isycos_drop_series(ctx, ys)


@pytest.mark.parametrize("extra", [dict(mode=0, pruning=1), dict(mode=1, pruning=1),
                                   dict(mode=1, pruning=0, chunks=3)],
                         ids=lambda d: ",".join("%s=%s" % kv for kv in d.items()))
def test_search_with_estimator1_matches_oracle(ctx, extra):
    api = _api()
    x, y = synth.planted_small_pair()
    kw = dict(k=4, s_min=32, s_max=256, sigma=0.2, seed=13, estimator=1)
    kw.update(extra)
    xs, ys = api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)
    api.isycos_reset_stats(ctx)
    got = api.isycos_search(ctx, xs, ys, 0, len(x), kw)
    st = api.isycos_get_stats(ctx)
    okw = dict(kw)
    mode = okw.pop("mode")
    if "chunks" in okw:
        ref, n = O.search_chunked(x, y, mode=mode, **okw)
    else:
        ref, n = (O.search_td if mode == 0 else O.search_bu)(x, y, **okw)
    _same(got, ref)
    assert st["decided_windows"] == n
    api.isycos_drop_series(ctx, xs)
    api.isycos_drop_series(ctx, ys)


def test_speculation_depth_changes_work_not_results(ctx):
    """ISYCOS_OPT_SPECULATION sets how many later BU climbs are asked ahead; the windows and
    the decided-window count stay those of the oracle for every depth."""
    api = _api()
    x, y = synth.planted_small_pair()
    kw = dict(k=4, s_min=32, s_max=256, sigma=0.2, pruning=1, seed=31, mode=1)
    xs, ys = api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)
    okw = dict(kw)
    okw.pop("mode")
    ref, n = O.search_bu(x, y, **okw)
    launches = {1: {}, 0: {}}
    try:
        for dev in (1, 0):   # the device-resident search, then the host machines
            api.isycos_set_option(ctx, api.OPT_BU_DEVICE, dev)
            for depth in (0, 1, 3, 8, 16, 24, 64):
                api.isycos_set_option(ctx, api.OPT_SPECULATION, depth)
                api.isycos_reset_stats(ctx)
                got = api.isycos_search(ctx, xs, ys, 0, len(x), kw)
                st = api.isycos_get_stats(ctx)
                _same(got, ref)
                assert st["decided_windows"] == n
                launches[dev][depth] = st["launches"]
    finally:
        api.isycos_set_option(ctx, api.OPT_SPECULATION, 24)   # the default
        api.isycos_set_option(ctx, api.OPT_BU_DEVICE, 0)
    assert launches[0][3] < launches[0][0]                  # host: fewer round trips
    assert all(v == 1 for v in launches[1].values())        # device: one launch
    api.isycos_drop_series(ctx, xs)
    api.isycos_drop_series(ctx, ys)


def test_serving_mixed_kinds_of_query(ctx):
    """Served queries of every kind at once (TD, BU, selection, chunked, estimator 1), each
    with its own parameters, return what the same query returns alone."""
    api = _api()
    pairs = []
    for p in range(3):
        x, y, _ = synth.planted_pair(4, 20 + p, 8000, len_lo=50, len_hi=1500)
        pairs.append((api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)))
    kinds = [dict(mode=0, pruning=1), dict(mode=1, pruning=1, seed=3),
             dict(mode=2, sel_partitions=8, sel_samples=3, seed=5), dict(mode=1, chunks=4),
             dict(mode=0, estimator=1), dict(mode=1, estimator=1, pruning=1)]
    jobs = []
    for i, kind in enumerate(kinds * 2):
        a, b = pairs[i % 3]
        prm = dict(k=4, s_min=32, s_max=400, **kind)
        jobs.append(((a, b, 100 * i, 8000 - 50 * i), prm))
    tickets = [api.isycos_serve_submit(ctx, *q, prm) for q, prm in jobs]
    res = {}
    deadline = time.time() + 300
    while len(res) < len(tickets) and time.time() < deadline:
        for t in tickets:
            if t not in res:
                r = api.isycos_serve_poll(ctx, t)
                if r is not None:
                    res[t] = r
        time.sleep(0.002)
    assert len(res) == len(tickets)
    for (q, prm), t in zip(jobs, tickets):
        assert np.array_equal(api.isycos_search(ctx, *q, prm), res[t][0])


def test_one_call_mixing_k_and_estimators(ctx):
    """Queries with different k and estimators in one call (one lane, so that one round
    carries several batches): every query returns what it returns alone."""
    api = _api()
    x, y = synth.planted_small_pair()
    xs, ys = api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)
    qs = [(xs, ys, 0, len(x), dict(k=k, s_min=32, s_max=256, mode=mode, estimator=est, pruning=1, seed=2))
          for k in (3, 4) for est in (0, 1) for mode in (0, 1)]
    alone = [api.isycos_search(ctx, *q[:4], q[4]) for q in qs]
    try:
        for lanes in (1, 3):
            api.isycos_set_option(ctx, api.OPT_LANES, lanes)
            got = api.isycos_search_queries(ctx, qs)
            for a, g in zip(alone, got):
                assert np.array_equal(a, g), lanes
    finally:
        api.isycos_set_option(ctx, api.OPT_LANES, 12)
    api.isycos_drop_series(ctx, xs)
    api.isycos_drop_series(ctx, ys)


def test_series_added_while_queries_are_served(ctx):
    """The caller may add series while served queries run (the library's serving threads
    read the series tables concurrently); every result still equals the query alone."""
    api = _api()
    x, y, _ = synth.planted_pair(4, 40, 20000, len_lo=50, len_hi=2000)
    xs, ys = api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)
    prm = dict(k=4, s_min=32, s_max=512, mode=1, pruning=1, seed=4)
    qs = [(xs, ys, 1000 * i, 20000 - 500 * i) for i in range(8)]
    tickets = [api.isycos_serve_submit(ctx, *q, prm) for q in qs]
    extra = []
    for i in range(300):   # grows the series tables while the queries run
        z = synth.normal(synth.seed_for(41, i), 64).astype(np.float32)
        extra.append(api.isycos_put_series(ctx, z))
    res = {}
    deadline = time.time() + 300
    while len(res) < len(tickets) and time.time() < deadline:
        for t in tickets:
            if t not in res:
                r = api.isycos_serve_poll(ctx, t)
                if r is not None:
                    res[t] = r
        time.sleep(0.002)
    assert len(res) == len(tickets)
    for q, t in zip(qs, tickets):
        assert np.array_equal(api.isycos_search(ctx, *q, prm), res[t][0])
    for e in extra:
        api.isycos_drop_series(ctx, e)


@pytest.mark.parametrize("extra", PARAMS[2:4] + PARAMS[5:6] + PARAMS[7:8],
                         ids=lambda d: ",".join("%s=%s" % kv for kv in d.items()))
def test_bu_on_the_device_and_on_the_host_match_oracle(ctx, extra):
    """SYCOS_BU with every decision on the device (one launch per call) and with the host
    search machines (one launch per round): both equal the oracle, with the same
    decided-window counts."""
    api = _api()
    x, y = synth.planted_small_pair()
    kw = dict(k=4, s_min=32, s_max=256, sigma=0.2, seed=11)
    kw.update(extra)
    ref, n = O.search_bu(x, y, **{k: v for k, v in kw.items() if k != "mode"})
    xs, ys = api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)
    try:
        for dev in (1, 0):
            api.isycos_set_option(ctx, api.OPT_BU_DEVICE, dev)
            api.isycos_reset_stats(ctx)
            got = api.isycos_search(ctx, xs, ys, 0, len(x), kw)
            st = api.isycos_get_stats(ctx)
            _same(got, ref)
            assert st["decided_windows"] == n, (dev, st["decided_windows"], n)
            if dev:
                assert st["launches"] == 1
    finally:
        api.isycos_set_option(ctx, api.OPT_BU_DEVICE, 0)
    api.isycos_drop_series(ctx, xs)
    api.isycos_drop_series(ctx, ys)


def test_device_search_time_limit_returns_timeout(ctx):
    """A device-resident search that runs past its time limit stops between rounds and the
    call returns ISYCOS_E_TIMEOUT; the context stays usable and the next call (no limit)
    returns the oracle's windows."""
    api = _api()
    x, y, _ = synth.planted_pair(2, 3, 60000)
    xs, ys = api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)
    kw = dict(k=4, s_min=32, s_max=1024, sigma=0.2, pruning=1, seed=5, mode=1)
    api.isycos_set_option(ctx, api.OPT_BU_DEVICE, 1)
    try:
        api.isycos_set_option(ctx, api.OPT_TIME_LIMIT_MS, 1)
        with pytest.raises(api.IsycosError) as e:
            api.isycos_search(ctx, xs, ys, 0, len(x), kw)
        assert e.value.status == api.E_TIMEOUT
        api.isycos_set_option(ctx, api.OPT_TIME_LIMIT_MS, 60000)
        got = api.isycos_search(ctx, xs, ys, 0, len(x), kw)
    finally:
        api.isycos_set_option(ctx, api.OPT_TIME_LIMIT_MS, 60000)
        api.isycos_set_option(ctx, api.OPT_BU_DEVICE, 0)
    ref, _ = O.search_bu(x, y, **{k: v for k, v in kw.items() if k != "mode"})
    _same(got, ref)
    api.isycos_drop_series(ctx, xs)
    api.isycos_drop_series(ctx, ys)
