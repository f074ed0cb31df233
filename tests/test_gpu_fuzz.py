"""Seeded randomised parity (GPU): searches and window batches over random parameter
combinations against the oracle, to catch interactions that the targeted tests miss
(several k and estimators in one call, chunked selection, tied data, odd window sizes)."""
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


def _series(rng, n, case):
    s = synth.seed_for(300, case)
    x, y, _ = synth.planted_pair(5, case, n, len_lo=40, len_hi=max(60, n // 3))
    kind = case % 3
    if kind == 1:   # heavy ties
        x, y = synth.quantize(x, 2.0), synth.quantize(y, 2.0)
    elif kind == 2:   # uniform noise with duplicated stretches
        x = synth.uniform(s, n).astype(np.float32)
        y = synth.uniform(s ^ 7, n).astype(np.float32)
        x[n // 3: n // 3 + 40] = x[n // 3]
        y[n // 3: n // 3 + 40] = y[n // 3]
    return np.ascontiguousarray(x, np.float32), np.ascontiguousarray(y, np.float32)


def _params(rng):
    k = int(rng.integers(1, 9))
    s_min = int(rng.integers(k + 1, 48))
    s_max = int(rng.integers(s_min, 320))
    p = dict(k=k, s_min=s_min, s_max=s_max, sigma=float(rng.choice([0.15, 0.2, 0.3])),
             pruning=int(rng.integers(0, 2)), seed=int(rng.integers(0, 1 << 30)),
             estimator=int(rng.integers(0, 2)), score_kind=int(rng.integers(0, 2)))
    if p["score_kind"] == 1:
        p["sigma"] = float(rng.choice([0.3, 0.5]))
    if rng.random() < 0.3:
        p["delta_td"] = int(rng.integers(k + 1, max(k + 2, s_min)))
    if rng.random() < 0.3:
        p["delta_bu"] = int(rng.integers(1, max(2, s_min // 2)))
    if rng.random() < 0.3:
        p["t_max_idle"] = int(rng.integers(0, 5))
    return p


def _oracle(x, y, q, prm):
    okw = dict(prm)
    mode = okw.pop("mode")
    chunks = okw.pop("chunks", 0)
    tb, te = q
    if mode == 2:
        return O.search_auto(x, y, t_begin=tb, t_end=te, partitions=okw.pop("sel_partitions"),
                             samples=okw.pop("sel_samples"), chunks=chunks, **okw)[:2]
    if chunks > 1:
        return O.search_chunked(x, y, t_begin=tb, t_end=te, mode=mode, chunks=chunks, **okw)
    return (O.search_td if mode == 0 else O.search_bu)(x, y, t_begin=tb, t_end=te, **okw)


def test_random_searches_in_one_call_match_the_oracle(ctx):
    api = _api()
    rng = np.random.default_rng(2024)
    data, queries, expect = [], [], []
    for case in range(30):
        n = int(rng.integers(600, 2400))
        x, y = _series(rng, n, case)
        xs, ys = api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)
        data.append((xs, ys))
        prm = _params(rng)
        prm["mode"] = int(rng.integers(0, 3))
        if prm["mode"] == 2:
            prm.update(sel_partitions=int(rng.integers(3, 10)), sel_samples=int(rng.integers(1, 4)))
        if rng.random() < 0.3:
            prm["chunks"] = int(rng.integers(2, 5))
        tb = int(rng.integers(0, n // 4))
        te = int(rng.integers(3 * n // 4, n + 1))
        queries.append((xs, ys, tb, te, prm))
        expect.append(_oracle(x, y, (tb, te), prm))
    api.isycos_reset_stats(ctx)
    got = api.isycos_search_queries(ctx, queries)
    st = api.isycos_get_stats(ctx)
    for i, (g, (ref, n_eval)) in enumerate(zip(got, expect)):
        gw = [(int(a), int(b)) for a, b in zip(g["t_s"], g["t_e"])]
        assert gw == [(a, b) for a, b, _, _ in ref], (i, queries[i][4])
        for (a, b, sc, mi), gs, gm in zip(ref, g["score"], g["mi"]):
            assert abs(gs - sc) <= 1e-12 and abs(gm - mi) <= 1e-12, (i, queries[i][4])
    assert st["decided_windows"] == sum(n for _, n in expect)
    for xs, ys in data:
        api.isycos_drop_series(ctx, xs)
        api.isycos_drop_series(ctx, ys)


@pytest.mark.parametrize("estimator", [0, 1])
def test_random_window_batches_match_the_oracle(ctx, estimator):
    """Random window lists (sizes k+1..6000, every path and bucket in one launch, tied and
    untied data): per-window integer sums against the oracle on every window."""
    api = _api()
    rng = np.random.default_rng(77 + estimator)
    n = 20000
    for case in range(3):
        x, y = _series(rng, n, 10 + case)
        xs, ys = api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)
        k = int(rng.integers(1, 9))
        sizes = np.concatenate([rng.integers(k + 1, 70, 40), rng.integers(70, 1100, 25),
                                rng.integers(1100, 6000, 4)])
        starts = np.array([int(rng.integers(0, n - m)) for m in sizes])
        w = api.windows_array(xs, ys, starts, sizes)
        api.isycos_set_option(ctx, api.OPT_ESTIMATOR, estimator)
        try:
            got = {}
            for opt in (0, 1, 2):
                api.isycos_set_option(ctx, api.OPT_KERNEL, opt)
                got[opt] = api.isycos_mi_windows(ctx, w, k)
        finally:
            api.isycos_set_option(ctx, api.OPT_KERNEL, 0)
            api.isycos_set_option(ctx, api.OPT_ESTIMATOR, 0)
        for opt in (1, 2):
            assert np.array_equal(got[0]["s_psi"], got[opt]["s_psi"]), (case, opt)
        for i, (s, m) in enumerate(zip(starts, sizes)):
            r = O.ksg_window(x[s:s + m], y[s:s + m], k, points=False, estimator=estimator)
            assert got[0]["s_psi"][i] == r["s_psi"] and got[0]["s_log"][i] == r["s_log"], (case, i, m, k)
            assert got[0]["mi"][i] == r["mi"] and got[0]["nmi"][i] == r["nmi"], (case, i, m, k)
        api.isycos_drop_series(ctx, xs)
        api.isycos_drop_series(ctx, ys)
