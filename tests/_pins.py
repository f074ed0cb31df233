"""Pins of the CPU oracle against what arXiv 2204.09131 and the mathematics fix.

Each ``pin_*`` function raises AssertionError when the oracle disagrees with a fact that
does not come from the oracle itself:

- ``pin_paper_example``: the neighbour sets and counts stated for the 7-point example of
  Sec. 7.1 (tests/golden/box_assisted_example_sec7.txt);
- ``pin_hand_window``: a 4-point window whose counts are worked by hand below;
- ``pin_brute_force``: an independent NumPy brute force (full lexicographic sort of
  (d_ij, j), binary32 distances) and SciPy's digamma on small windows with and without ties;
- ``pin_closed_form``: Y = X, Y = -X and Y = 2^s X, where every marginal count equals k
  and Eq. KSGmi reduces to psi(m) - psi(k) - 1/k (SciPy digamma);
- ``pin_entropy``: the plug-in joint entropy against SciPy's entropy of the cell counts;
- ``pin_invariants``: symmetry, sign and power-of-two scale invariance, bit for bit;
- ``pin_gaussian``: the bivariate-Gaussian closed form -1/2 ln(1 - rho^2) within the
  estimator's sampling error;
- ``pin_est1_*``: the same kinds of pins for Kraskov's first estimator (strict counts in
  strips of half-width eps_i, psi(n + 1), no -1/k): a hand-worked window, the NumPy brute
  force, and the closed form Y = X, where every count is k - 1 and the estimate is
  psi(m) - psi(k).

The same functions run against planted mistakes of the oracle (tests/test_oracle_mutations.py)
to show that each plausible mistake fails at least one pin.
"""
from __future__ import annotations

import math
import os

import numpy as np
from scipy.special import digamma
from scipy.stats import entropy

from oracle import oracle as O
from paper_2204_09131_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ---------------------------------------------------------------------------
# Independent NumPy brute force (test-local; shares nothing with the oracle's C code)
# ---------------------------------------------------------------------------

def numpy_ksg(x, y, k):
    x = np.asarray(x, dtype=np.float32)
    y = np.asarray(y, dtype=np.float32)
    m = x.shape[0]
    ax = np.abs(x[:, None] - x[None, :])          # binary32 differences
    ay = np.abs(y[:, None] - y[None, :])
    d = np.maximum(ax, ay)
    nx = np.empty(m, dtype=np.int64)
    ny = np.empty(m, dtype=np.int64)
    c = np.empty(m, dtype=np.int64)
    for i in range(m):
        js = np.array([j for j in range(m) if j != i])
        order = np.lexsort((js, d[i, js]))        # by distance, then by index
        knn = js[order[:k]]
        dx = ax[i, knn].max()
        dy = ay[i, knn].max()
        nx[i] = int(np.sum(ax[i, js] <= dx))
        ny[i] = int(np.sum(ay[i, js] <= dy))
        c[i] = int(np.sum((x == x[i]) & (y == y[i])))
    mi = digamma(k) - 1.0 / k - np.mean(digamma(nx) + digamma(ny)) + digamma(m)
    h = math.log(m) - np.mean(np.log(c))
    return nx, ny, c, mi, h


def numpy_ksg1(x, y, k):
    """Kraskov's first estimator by brute force: eps_i = k-th smallest max-norm distance to
    the other points, n_x = #{j != i : |x_i - x_j| < eps_i}, psi(k) + psi(m) - <psi(n_x + 1)
    + psi(n_y + 1)>."""
    x = np.asarray(x, dtype=np.float32)
    y = np.asarray(y, dtype=np.float32)
    m = x.shape[0]
    ax = np.abs(x[:, None] - x[None, :])
    ay = np.abs(y[:, None] - y[None, :])
    d = np.maximum(ax, ay)
    nx = np.empty(m, dtype=np.int64)
    ny = np.empty(m, dtype=np.int64)
    for i in range(m):
        others = np.delete(np.arange(m), i)
        eps = np.sort(d[i, others])[k - 1]
        nx[i] = int(np.sum(ax[i, others] < eps))
        ny[i] = int(np.sum(ay[i, others] < eps))
    mi = digamma(k) + digamma(m) - np.mean(digamma(nx + 1) + digamma(ny + 1))
    return nx, ny, mi


# ---------------------------------------------------------------------------
# Pins
# ---------------------------------------------------------------------------

def load_paper_example():
    pts = {}
    expect = None
    with open(os.path.join(GOLDEN, "box_assisted_example_sec7.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == "expect":
                kv = dict(p.split("=") for p in parts[3:])
                expect = {"k": int(parts[1]), "point": parts[2], **kv}
            else:
                pts[parts[0]] = (float(parts[1]), float(parts[2]))
    return pts, expect


def pin_paper_example():
    pts, ex = load_paper_example()
    names = list(pts)
    x = np.array([pts[n][0] for n in names], dtype=np.float32)
    y = np.array([pts[n][1] for n in names], dtype=np.float32)
    i = names.index(ex["point"])
    k = ex["k"]
    r = O.ksg_window(x, y, k)
    assert r["nx"][i] == int(ex["nx"]), ("n_x of p1", r["nx"][i])
    assert r["ny"][i] == int(ex["ny"]), ("n_y of p1", r["ny"][i])
    # The strips themselves: members counted by the paper, recomputed from the oracle's
    # per-dimension distances.
    xs = sorted(n for j, n in enumerate(names) if j != i and abs(x[j] - x[i]) <= r["dx"][i])
    ys = sorted(n for j, n in enumerate(names) if j != i and abs(y[j] - y[i]) <= r["dy"][i])
    assert xs == sorted(ex["xstrip"].split(",")), xs
    assert ys == sorted(ex["ystrip"].split(",")), ys
    # The k-th neighbour distance is that of p3, the farther of the two stated neighbours.
    knn = ex["knn"].split(",")
    d = [max(abs(x[names.index(n)] - x[i]), abs(y[names.index(n)] - y[i])) for n in knn]
    assert r["eps"][i] == np.float32(max(d)), (r["eps"][i], d)


def pin_hand_window():
    # p0=(0,0) p1=(1,.5) p2=(3,0) p3=(3.5,2), k=1, max-norm distances:
    # d01=1 d02=3 d03=3.5 d12=2 d13=2.5 d23=2.
    # p0: NN p1 -> dx=1 dy=.5 -> n_x={p1}=1, n_y={p1,p2}=2
    # p1: NN p0 -> dx=1 dy=.5 -> n_x={p0}=1, n_y={p0,p2}=2
    # p2: d21=d23=2, tie broken toward the smaller index -> NN p1 -> dx=2 dy=.5
    #     -> n_x={p1,p3}=2, n_y={p0,p1}=2
    # p3: NN p2 -> dx=.5 dy=2 -> n_x={p2}=1, n_y={p0,p1,p2}=3
    x = np.array([0.0, 1.0, 3.0, 3.5], dtype=np.float32)
    y = np.array([0.0, 0.5, 0.0, 2.0], dtype=np.float32)
    r = O.ksg_window(x, y, 1)
    assert list(r["nx"]) == [1, 1, 2, 1], r["nx"]
    assert list(r["ny"]) == [2, 2, 2, 3], r["ny"]
    assert list(r["c"]) == [1, 1, 1, 1], r["c"]
    mi = digamma(1) - 1.0 + digamma(4) - (
        (digamma(1) + digamma(2)) * 2 + (digamma(2) + digamma(2)) + (digamma(1) + digamma(3))) / 4
    assert abs(r["mi_exact"] - mi) < 1e-12, (r["mi_exact"], mi)
    assert abs(r["mi"] - mi) < 1e-8, (r["mi"], mi)


def _small_cases():
    cases = []
    for t, (m, k) in enumerate([(5, 1), (9, 2), (17, 3), (40, 4), (64, 6), (100, 4), (33, 8)]):
        s = synth.seed_for(90, t)
        x = synth.normal(s, m).astype(np.float32)
        y = (0.7 * synth.normal(s ^ 1, m) + 0.3 * x).astype(np.float32)
        cases.append((x, y, k))
        # heavy ties: quantised to a coarse grid (duplicates of (x, y) included)
        cases.append((synth.quantize(x, 2.0), synth.quantize(y, 2.0), k))
    # all points identical but one
    cases.append((np.array([1, 1, 1, 1, 1, 2], np.float32), np.array([0, 0, 0, 0, 0, 1], np.float32), 2))
    return cases


def pin_brute_force():
    for x, y, k in _small_cases():
        nx, ny, c, mi, h = numpy_ksg(x, y, k)
        r = O.ksg_window(x, y, k)
        assert np.array_equal(r["nx"], nx), (k, r["nx"], nx)
        assert np.array_equal(r["ny"], ny), (k, r["ny"], ny)
        assert np.array_equal(r["c"], c), (k, r["c"], c)
        assert abs(r["mi_exact"] - mi) < 1e-10, (r["mi_exact"], mi)
        assert abs(r["mi"] - mi) < 1e-8, (r["mi"], mi)
        assert abs(r["h_exact"] - h) < 1e-10, (r["h_exact"], h)


def _tie_free_line(x, k):
    """True when, for every i, the k-th and (k+1)-th smallest |x_i - x_j| differ."""
    x = np.asarray(x, dtype=np.float32)
    ax = np.abs(x[:, None] - x[None, :])
    np.fill_diagonal(ax, np.inf)
    s = np.sort(ax, axis=1)
    return bool(np.all(s[:, k - 1] < s[:, k]))


def pin_closed_form():
    for t, (m, k) in enumerate([(32, 4), (64, 3), (128, 6), (257, 4), (40, 1)]):
        x = synth.normal(synth.seed_for(91, t), m).astype(np.float32)
        assert _tie_free_line(x, k)
        expect = digamma(m) - digamma(k) - 1.0 / k
        for y in (x.copy(), -x, np.float32(4.0) * x, np.float32(0.125) * x):
            r = O.ksg_window(x, y, k)
            assert np.all(r["nx"] == k) and np.all(r["ny"] == k), (r["nx"], r["ny"])
            assert abs(r["mi_exact"] - expect) < 1e-11, (r["mi_exact"], expect)
            assert abs(r["mi"] - expect) < 1e-8, (r["mi"], expect)


def pin_entropy():
    for t, m in enumerate([50, 120]):
        s = synth.seed_for(92, t)
        x = synth.quantize(synth.normal(s, m), 2.0)
        y = synth.quantize(synth.normal(s ^ 3, m), 2.0)
        r = O.ksg_window(x, y, 3)
        _, counts = np.unique(np.stack([x, y], 1), axis=0, return_counts=True)
        h = entropy(counts / m)                    # natural log
        assert abs(r["h_exact"] - h) < 1e-12, (r["h_exact"], h)
        assert abs(r["h_w"] - h) < 1e-8, (r["h_w"], h)
        assert abs(r["nmi"] - r["mi"] / r["h_w"]) < 1e-15
        # tie-free: H = ln m
        xf = synth.normal(s ^ 5, m).astype(np.float32)
        r2 = O.ksg_window(xf, xf[::-1].copy(), 3)
        assert abs(r2["h_exact"] - math.log(m)) < 1e-12


def pin_invariants():
    for t, (m, k) in enumerate([(64, 4), (200, 3), (96, 6)]):
        s = synth.seed_for(93, t)
        x, y = synth.gaussian_pair(s, m, 0.5)
        base = O.ksg_window(x, y, k)
        for xx, yy in ((y, x), (-x, y), (x, -y), (x * np.float32(8.0), y * np.float32(8.0))):
            r = O.ksg_window(xx, yy, k)
            assert r["s_psi"] == base["s_psi"] and r["mi"] == base["mi"], (r["mi"], base["mi"])
        perm = np.argsort(synth.uniform(s ^ 9, m))
        r = O.ksg_window(x[perm], y[perm], k)
        assert r["s_psi"] == base["s_psi"]


def pin_gaussian(windows=24, m=256, estimator=0):
    for t, rho in enumerate([0.0, 0.6, 0.9]):
        vals = []
        for w in range(windows):
            x, y = synth.gaussian_pair(synth.seed_for(94, t, w), m, rho)
            vals.append(O.ksg_window(x, y, 4, points=False, estimator=estimator)["mi_exact"])
        vals = np.array(vals)
        truth = -0.5 * math.log(1.0 - rho * rho)
        se = vals.std(ddof=1) / math.sqrt(len(vals))
        # 4 standard errors plus a small-sample bias margin of the estimator
        assert abs(vals.mean() - truth) < 4.0 * se + 0.03, (rho, vals.mean(), truth, se)


def pin_est1_hand_window():
    # The window of pin_hand_window, k = 1, Kraskov's first estimator:
    # p0: eps=1 (p1); |dx|<1: none -> n_x=0; |dy|<1: p1 (.5), p2 (0) -> n_y=2
    # p1: eps=1 (p0); |dx|<1: none -> 0;      |dy|<1: p0 (.5), p2 (.5) -> 2
    # p2: eps=2 (p1, p3); |dx|<2: p3 (.5) -> 1 (p1 at exactly 2 is out); |dy|<2: p0, p1 -> 2
    # p3: eps=2 (p2); |dx|<2: p2 (.5) -> 1;   |dy|<2: p1 (1.5) -> 1
    x = np.array([0.0, 1.0, 3.0, 3.5], dtype=np.float32)
    y = np.array([0.0, 0.5, 0.0, 2.0], dtype=np.float32)
    r = O.ksg_window(x, y, 1, estimator=1)
    assert list(r["nx"]) == [0, 0, 1, 1], r["nx"]
    assert list(r["ny"]) == [2, 2, 2, 1], r["ny"]
    mi = digamma(1) + digamma(4) - (
        2 * (digamma(1) + digamma(3)) + (digamma(2) + digamma(3)) + (digamma(2) + digamma(2))) / 4
    assert abs(r["mi_exact"] - mi) < 1e-12, (r["mi_exact"], mi)
    assert abs(r["mi"] - mi) < 1e-8, (r["mi"], mi)


def pin_est1_brute_force():
    for x, y, k in _small_cases():
        nx, ny, mi = numpy_ksg1(x, y, k)
        r = O.ksg_window(x, y, k, estimator=1)
        assert np.array_equal(r["nx"], nx), (k, r["nx"], nx)
        assert np.array_equal(r["ny"], ny), (k, r["ny"], ny)
        assert abs(r["mi_exact"] - mi) < 1e-10, (r["mi_exact"], mi)
        assert abs(r["mi"] - mi) < 1e-8, (r["mi"], mi)
        base = O.ksg_window(x, y, k)
        assert np.array_equal(r["c"], base["c"]) and r["h_w"] == base["h_w"]


def pin_est1_closed_form():
    for t, (m, k) in enumerate([(32, 4), (64, 3), (128, 6), (257, 4), (40, 1)]):
        x = synth.normal(synth.seed_for(91, t), m).astype(np.float32)
        assert _tie_free_line(x, k)
        expect = digamma(m) - digamma(k)
        # (the strips have the same half-width in both dimensions, so unlike the second
        # estimator a scaled Y = 2^s X does not reduce to the closed form)
        for y in (x.copy(), -x):
            r = O.ksg_window(x, y, k, estimator=1)
            assert np.all(r["nx"] == k - 1) and np.all(r["ny"] == k - 1), (r["nx"], r["ny"])
            assert abs(r["mi_exact"] - expect) < 1e-11, (r["mi_exact"], expect)
            assert abs(r["mi"] - expect) < 1e-8, (r["mi"], expect)
            sym = O.ksg_window(y, x, k, estimator=1)
            assert sym["mi"] == r["mi"]


FAST_PINS = [pin_paper_example, pin_hand_window, pin_brute_force, pin_closed_form,
             pin_entropy, pin_invariants, pin_est1_hand_window, pin_est1_brute_force,
             pin_est1_closed_form]
