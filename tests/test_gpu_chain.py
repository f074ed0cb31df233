"""Incremental window MI (Sec. 7.1 influenced regions, Lemmas 3-6) against from-scratch (GPU).

isycos_mi_chain derives each window's neighbour state from the previous window's; its
results must equal isycos_mi_windows (integer sums bit-exact, scalars identical) and the
oracle, for sliding (TD), ring-walking (BU), growing, shrinking and jumping sequences, with
and without ties -- and it must actually skip work when the step is small.
"""
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


def _compare(ctx, xs, ys, starts, sizes, k, x=None, y=None, oracle_every=0):
    api = _api()
    inc = api.isycos_mi_chain(ctx, xs, ys, starts, sizes, k)
    ref = api.isycos_mi_windows(ctx, api.windows_array(xs, ys, starts, sizes), k)
    assert np.array_equal(inc["s_psi"], ref["s_psi"]), np.nonzero(inc["s_psi"] != ref["s_psi"])
    assert np.array_equal(inc["s_log"], ref["s_log"])
    assert np.array_equal(inc["mi"], ref["mi"]) and np.array_equal(inc["nmi"], ref["nmi"])
    if oracle_every:
        for i in range(0, len(starts), oracle_every):
            s, m = int(starts[i]), int(sizes[i])
            r = O.ksg_window(x[s:s + m], y[s:s + m], k, points=False)
            assert inc["s_psi"][i] == r["s_psi"] and inc["mi"][i] == r["mi"]
    return inc


@pytest.mark.parametrize("m,delta", [(64, 1), (64, 16), (256, 3), (1000, 8), (1000, 250), (4096, 32)])
def test_sliding_chain(ctx, m, delta):
    api = _api()
    n = 20000
    x, y, _ = synth.planted_pair(7, m, n)
    xs, ys = api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)
    starts = np.arange(0, min(n - m, 60 * delta + 1), delta)
    _compare(ctx, xs, ys, starts, np.full(len(starts), m), 4, x, y, oracle_every=17)


def test_sliding_chain_saves_work(ctx):
    api = _api()
    n = 30000
    x, y, _ = synth.planted_pair(7, 1, n)
    xs, ys = api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)
    starts = np.arange(0, 200 * 4, 4)
    api.isycos_reset_stats(ctx)
    api.isycos_mi_chain(ctx, xs, ys, starts, np.full(len(starts), 2048), 4)
    st = api.isycos_get_stats(ctx)
    total = 2048 * len(starts)
    # each segment of at least 16 windows starts from scratch (2048 points); after that, a
    # step of 4 points re-searches only the points whose influenced region holds a removed
    # or added point
    assert st["incr_windows"] == len(starts)
    n_seg = -(-len(starts) // 16)
    assert st["incr_full_points"] < n_seg * 2048 + 0.05 * total, st


@pytest.mark.parametrize("k", [1, 4, 6])
def test_ring_walk_chain(ctx, k):
    """A BU step: the current window, then its ring N_r walked along the perimeter."""
    api = _api()
    n = 12000
    x, y, _ = synth.planted_pair(7, 20 + k, n)
    xs, ys = api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)
    ts, te, d = 5000, 5600, 8
    starts, sizes = [ts], [te - ts + 1]
    for r in (1, 2, 3):
        ring = []
        for a in range(-r, r + 1):
            for b in range(-r, r + 1):
                if max(abs(a), abs(b)) == r:
                    ring.append((a, b))
        # perimeter order: sort by angle so that consecutive windows differ by one step
        ring.sort(key=lambda ab: np.arctan2(ab[1], ab[0]))
        for a, b in ring:
            starts.append(ts + a * d)
            sizes.append(te + b * d - (ts + a * d) + 1)
    _compare(ctx, xs, ys, np.array(starts), np.array(sizes), k, x, y, oracle_every=5)


def test_growing_shrinking_jumping_chain(ctx):
    api = _api()
    n = 60000
    x, y, _ = synth.planted_pair(7, 40, n)
    xs, ys = api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)
    starts, sizes = [], []
    s, m = 1000, 40
    rng = np.random.default_rng(2)
    for i in range(120):
        op = rng.integers(0, 5)
        if op == 0:
            m = min(m + int(rng.integers(1, 50)), 3000)        # grow right
        elif op == 1:
            g = int(rng.integers(1, 40)); s -= g; m += g       # grow left
        elif op == 2 and m > 60:
            m -= int(rng.integers(1, 20))                      # shrink right
        elif op == 3 and m > 60:
            g = int(rng.integers(1, 20)); s += g; m -= g       # shrink left
        else:
            s += int(rng.integers(-30, 30))                    # shift
        if i in (50, 90):
            s += 20000 if i == 50 else -15000                 # jump: no overlap
        s = max(0, min(s, n - m))
        starts.append(s)
        sizes.append(m)
    # windows larger than one ring can hold: a new chain starts at each of them
    starts += [30000, 38000, 39000]
    sizes += [10000, 10000, 12000]
    _compare(ctx, xs, ys, np.array(starts), np.array(sizes), 4, x, y, oracle_every=13)


def test_chain_with_ties_and_duplicates(ctx):
    api = _api()
    n = 8000
    x, y, _ = synth.planted_pair(7, 50, n)
    for step_inv in (10.0, 2.0, 1.0):
        xq, yq = synth.quantize(x, step_inv), synth.quantize(y, step_inv)
        xs, ys = api.isycos_put_series(ctx, xq), api.isycos_put_series(ctx, yq)
        starts = np.arange(100, 100 + 80 * 5, 5)
        _compare(ctx, xs, ys, starts, np.full(len(starts), 300), 3, xq, yq, oracle_every=9)
        starts2 = np.arange(3000, 3000 + 40 * 2, 2)
        _compare(ctx, xs, ys, starts2, np.full(len(starts2), 64), 6)
