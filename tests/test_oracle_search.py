"""The oracle's SYCOS_TD / SYCOS_BU (Algorithms 1 and 2, Sec. 6 pruning) on hand-traced
score tables and on the planted-segment pair (CPU only)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2204_09131_gb300 import synth
from tests import _search_pins


@pytest.mark.parametrize("pin", _search_pins.SEARCH_PINS, ids=lambda f: f.__name__)
def test_hand_traced_search(pin):
    """The hand traces of tests/_search_pins.py: which windows each search scores, in which
    order, and what it returns, on mocked score tables."""
    pin()


def _check_properties(wins, n, s_min, s_max, sigma):
    prev_end = -1
    for ts, te, sc, _ in wins:
        assert ts > prev_end and te >= ts
        assert s_min <= te - ts + 1 <= s_max
        assert 0 <= ts and te < n
        assert sc >= sigma
        prev_end = te


@pytest.mark.parametrize("search", ["td", "bu"])
@pytest.mark.parametrize("pruning", [0, 1])
def test_planted_pair_recovery(search, pruning):
    x, y = synth.planted_small_pair()
    fn = O.search_td if search == "td" else O.search_bu
    wins, _ = fn(x, y, k=4, s_min=32, s_max=256, sigma=0.2, pruning=pruning, seed=11)
    _check_properties(wins, len(x), 32, 256, 0.2)
    hit_a = any(ts < 700 and te >= 400 for ts, te, _, _ in wins)
    hit_b = any(ts < 1500 and te >= 1200 for ts, te, _, _ in wins)
    assert hit_a and hit_b, wins
    # Windows found away from the planted segments are rare on this seed.
    outside = [w for w in wins if w[1] < 380 or (w[0] > 720 and w[1] < 1180) or w[0] > 1520]
    assert len(outside) <= 1, outside


def test_bu_lahc_index_stream():
    # The history index of step s of climb c is SplitMix64 output (c << 32) + s + 1 mod h.
    seed = 99
    v = [O.splitmix64_at(seed, (2 << 32) + s + 1) % 8 for s in range(5)]
    assert all(0 <= a < 8 for a in v)
    assert v == [int(z) % 8 for z in synth.splitmix64(seed, 5, offset=(2 << 32))]


def test_invalid_params():
    x, y = synth.planted_small_pair(200)
    with pytest.raises(ValueError):
        O.search_td(x, y, k=4, s_min=4, s_max=64)       # s_min < k + 1
    with pytest.raises(ValueError):
        O.search_bu(x, y, k=4, s_min=64, s_max=32)      # s_max < s_min


def test_selection_scores_follow_the_equations():
    # Eqs. normalizeruntime / normalizedwindows / normalizedeffscore (Sec. 5.3) by hand:
    # t_TD = 100, t_BU = 300 -> t~ = 0.25, 0.75; nL_TD = 5, nS_BU = 2 -> n~ = 5/7, 2/7
    td, bu = O.nscores(100.0, 300.0, 5.0, 2.0, alpha=0.5)
    assert td == pytest.approx(0.5 * 4.0 + 0.5 * 5.0 / 7.0)
    assert bu == pytest.approx(0.5 / 0.75 + 0.5 * 2.0 / 7.0)
    # alpha = 1: runtime only; alpha = 0: window counts only
    assert O.nscores(1.0, 3.0, 0.0, 9.0, alpha=1.0) == pytest.approx((4.0, 4.0 / 3.0))
    assert O.nscores(1.0, 3.0, 1.0, 3.0, alpha=0.0) == pytest.approx((0.25, 0.75))
    # degenerate: nothing evaluated, nothing found
    assert O.nscores(0.0, 0.0, 0.0, 0.0, alpha=0.5) == pytest.approx((1.0, 1.0))


@pytest.mark.parametrize("seed", [1, 2])
def test_selection_runs_the_selected_search(seed):
    x, y = synth.planted_small_pair()
    kw = dict(k=4, s_min=32, s_max=256, sigma=0.2, pruning=1, seed=seed)
    wins, n, sel, sc = O.search_auto(x, y, partitions=10, samples=4, **kw)
    assert sel == (0 if sc[0] > sc[1] else 1)
    ref, _ = (O.search_td if sel == 0 else O.search_bu)(x, y, **kw)
    assert [(a, b) for a, b, _, _ in wins] == [(a, b) for a, b, _, _ in ref]
    assert n > 0


@pytest.mark.parametrize("mode", [0, 1])
def test_chunked_search_with_one_chunk_is_the_plain_search(mode):
    """Algorithm 4 with n_p = 1 is the unchunked search (a single chunk [0, N))."""
    x, y = synth.planted_small_pair()
    kw = dict(k=4, s_min=32, s_max=256, pruning=1, seed=3)
    plain = (O.search_td if mode == 0 else O.search_bu)(x, y, **kw)
    assert O.search_chunked(x, y, mode=mode, chunks=1, **kw) == plain


@pytest.mark.parametrize("mode", [0, 1])
def test_chunked_search_recovers_the_planted_segments(mode):
    """Chunks overlap by s_max, so segments that cross a chunk boundary are still found:
    with 4 chunks of 500 points the boundaries at 500 and 1500 cut both planted segments
    ([400, 700) and [1200, 1500)), and windows overlapping each are still returned."""
    x, y = synth.planted_small_pair()
    wins, _ = O.search_chunked(x, y, mode=mode, chunks=4, k=4, s_min=32, s_max=256, pruning=0)
    assert [w[0] for w in wins] == sorted(w[0] for w in wins)
    for lo, hi in ((400, 700), (1200, 1500)):
        assert any(a < hi and b >= lo for a, b, _, _ in wins), (lo, hi, wins)
    for a, b, sc, _ in wins:
        assert 0 <= a < b < len(x) and sc >= 0.2 and 32 <= b - a + 1 <= 256


def test_chunked_search_windows_lie_in_their_chunks():
    """Every returned window lies inside one chunk [i L - s_max, (i + 1) L) and no chunk's
    windows overlap each other (each chunk is a plain search); a mocked score that is high on
    one block only, far from the boundaries, gives exactly the unchunked windows."""
    def score(ts, te):
        inside = 300 <= ts and te < 500
        return (0.9 if inside else 0.0), 0.0
    N, chunks, s_max = 4000, 4, 128
    plain, _ = O.search_td(score, None, 0, N, k=4, s_min=32, s_max=s_max)
    chunked, _ = O.search_chunked(score, None, 0, N, mode=0, chunks=chunks, k=4, s_min=32, s_max=s_max)
    assert chunked == plain and plain
    L = N // chunks
    wins, _ = O.search_chunked(*synth.planted_small_pair(), mode=1, chunks=chunks, k=4,
                               s_min=32, s_max=s_max)
    for a, b, _, _ in wins:
        assert any(max(0, i - s_max) <= a and b < min(N, i + L) for i in range(0, N, L))
