"""Parity of the CUDA window-MI path with the CPU oracle (GPU).

The bar: per-point integers (n_x, n_y, c) and the integer sums S_psi, S_log bit-exact; the
binary64 scalars mi, h_w, nmi within 1e-12 (the path evaluates them in the same fixed order
from the same exact sums, so they agree to the last bit in practice; the tolerance stated
for these scalars is 1e-5).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2204_09131_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12


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


def _check_points(ctx, x, y, starts, sizes, k):
    api = _api()
    xs = api.isycos_put_series(ctx, x)
    ys = api.isycos_put_series(ctx, y)
    w = api.windows_array(xs, ys, starts, sizes)
    out, nx, ny, c = api.isycos_mi_windows_points(ctx, w, k)
    off = 0
    for i, (s, m) in enumerate(zip(starts, sizes)):
        r = O.ksg_window(x[s:s + m], y[s:s + m], k)
        assert np.array_equal(nx[off:off + m], r["nx"]), (m, k, "nx")
        assert np.array_equal(ny[off:off + m], r["ny"]), (m, k, "ny")
        assert np.array_equal(c[off:off + m], r["c"]), (m, k, "c")
        assert out["s_psi"][i] == r["s_psi"] and out["s_log"][i] == r["s_log"], (m, k)
        assert abs(out["mi"][i] - r["mi"]) <= TOL, (m, k, out["mi"][i], r["mi"])
        assert abs(out["h_w"][i] - r["h_w"]) <= TOL and abs(out["nmi"][i] - r["nmi"]) <= TOL
        off += m
    # the batched result without per-point outputs is the same
    out2 = api.isycos_mi_windows(ctx, w, k)
    assert np.array_equal(out2["s_psi"], out["s_psi"]) and np.array_equal(out2["mi"], out["mi"])
    api.isycos_drop_series(ctx, xs)
    api.isycos_drop_series(ctx, ys)
    return out


def test_tables_equal_the_oracle(ctx):
    api = _api()
    psi, lg = api.isycos_tables(ctx, api.MAX_M + 1)
    opsi, olg = O.fixed_tables(api.MAX_M + 1)
    assert np.array_equal(psi, opsi) and np.array_equal(lg, olg)


# sizes around every bucket edge and the 64-point block edge, plus a ragged tail
EDGE_SIZES = [5, 9, 31, 32, 33, 63, 64, 65, 100, 127, 128, 129, 255, 256, 257, 511, 513, 1000,
              2047, 2049]


@pytest.mark.parametrize("k", [1, 3, 4, 6, 8])
def test_points_bucket_edges(ctx, k):
    n = 6000
    x, y = synth.gaussian_pair(synth.seed_for(200, k), n, 0.5)
    sizes = [m for m in EDGE_SIZES if m >= k + 1]
    starts = [(97 * i) % (n - m) for i, m in enumerate(sizes)]
    _check_points(ctx, x, y, starts, sizes, k)


@pytest.mark.parametrize("k", [3, 4, 6])
def test_points_heavy_ties(ctx, k):
    # quantised to 0.1 (cfg 5 shape) and to a coarse 0.5 grid: many equal distances and
    # duplicate points, so the tie-break and the duplicate count matter
    n = 5000
    x, y = synth.gaussian_pair(synth.seed_for(201, k), n, 0.7)
    for step_inv in (10.0, 2.0):
        xq, yq = synth.quantize(x, step_inv), synth.quantize(y, step_inv)
        sizes = [k + 1, 33, 64, 200, 700, 1500]
        starts = [13 * i for i in range(len(sizes))]
        _check_points(ctx, xq, yq, starts, sizes, k)


def test_degenerate_windows(ctx):
    # all points identical; identical x only; identical y only; Y = X; Y = -X
    m = 150
    base = synth.normal(synth.seed_for(202, 0), m).astype(np.float32)
    cases = [(np.full(m, 1.5, np.float32), np.full(m, -2.0, np.float32)),
             (np.full(m, 3.0, np.float32), base),
             (base, np.zeros(m, np.float32)),
             (base, base.copy()),
             (base, -base)]
    for x, y in cases:
        _check_points(ctx, x, y, [0, 7], [m, m - 7], 4)


def test_closed_form_y_equals_x(ctx):
    api = _api()
    from scipy.special import digamma
    x = synth.normal(synth.seed_for(203, 0), 4096).astype(np.float32)
    out = _check_points(ctx, x, x.copy(), [0], [4096], 4)
    assert abs(out["mi"][0] - (digamma(4096) - digamma(4) - 0.25)) < 1e-8


def test_stride1_sweep_planted_pair(ctx):
    """Every window of size 32, 64 and 128 at stride 1 of the n = 2000 planted pair:
    5,779 windows (40,210,720 ordered pairs), bit-exact sums against the oracle."""
    api = _api()
    x, y = synth.planted_small_pair()
    wins = synth.stride_windows(len(x), [32, 64, 128])
    assert len(wins) == 5779
    xs = api.isycos_put_series(ctx, x)
    ys = api.isycos_put_series(ctx, y)
    w = api.windows_array(xs, ys, [s for s, _ in wins], [m for _, m in wins])
    assert int((w["m"].astype(np.int64) * (w["m"] - 1)).sum()) == 40210720
    out = api.isycos_mi_windows(ctx, w, 4)
    for i, (s, m) in enumerate(wins):
        r = O.ksg_window(x[s:s + m], y[s:s + m], 4, points=False)
        assert out["s_psi"][i] == r["s_psi"] and out["s_log"][i] == r["s_log"], (s, m)
        assert abs(out["mi"][i] - r["mi"]) <= TOL and abs(out["nmi"][i] - r["nmi"]) <= TOL
    # plain one-window-per-launch form gives the same results
    sub = w[::37]
    plain = api.isycos_mi_windows_plain(ctx, sub, 4)
    assert np.array_equal(plain["s_psi"], out["s_psi"][::37])
    assert np.array_equal(plain["mi"], out["mi"][::37])


def test_largest_windows_sampled_points(ctx):
    """Windows of the largest sizes (16384, 8192, 4096, 4095) in one batch, checked on sampled
    points (the oracle computes one point in O(m)) and, for m = 4096, on the whole window."""
    api = _api()
    n = 40000
    x, y, _ = synth.planted_pair(5, 0, n)
    xq, yq = synth.quantize(x), synth.quantize(y)
    for xx, yy in ((x, y), (xq, yq)):
        sizes = [16384, 8192, 4096, 4095, 64]
        starts = [0, 16384, 30000, 1234, 39000]
        xs = api.isycos_put_series(ctx, xx)
        ys = api.isycos_put_series(ctx, yy)
        w = api.windows_array(xs, ys, starts, sizes)
        out, nx, ny, c = api.isycos_mi_windows_points(ctx, w, 6)
        off = 0
        rng = np.random.default_rng(7)
        for s, m in zip(starts, sizes):
            pts = np.unique(np.concatenate([[0, m - 1], rng.integers(0, m, 40)]))
            for i in pts:
                r = O.ksg_point(xx[s:s + m], yy[s:s + m], 6, int(i))
                assert (nx[off + i], ny[off + i], c[off + i]) == (r["nx"], r["ny"], r["c"]), (m, i)
            off += m
        r = O.ksg_window(xx[30000:34096], yy[30000:34096], 6, points=False)
        assert out["s_psi"][2] == r["s_psi"] and abs(out["mi"][2] - r["mi"]) <= TOL
        api.isycos_drop_series(ctx, xs)
        api.isycos_drop_series(ctx, ys)


def test_device_path_matches_host_path(ctx):
    import torch
    api = _api()
    x, y, _ = synth.planted_pair(2, 1, 30000)
    xs = api.isycos_put_series(ctx, torch.from_numpy(x).cuda())
    ys = api.isycos_put_series(ctx, torch.from_numpy(y).cuda())
    rng = np.random.default_rng(3)
    sizes = rng.integers(5, 3000, 500)
    starts = [int(rng.integers(0, 30000 - m)) for m in sizes]
    w = api.windows_array(xs, ys, starts, sizes)
    host = api.isycos_mi_windows(ctx, w, 4)
    dw = torch.from_numpy(w.view(np.uint8)).cuda()
    dout = torch.empty(len(w) * 40, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    api.isycos_mi_windows_device(ctx, dw, len(w), 4, 3000, dout, st)
    api.isycos_device_status(ctx, st)
    dev = dout.cpu().numpy().view(api.MI_OUT_DTYPE)
    assert np.array_equal(dev["s_psi"], host["s_psi"]) and np.array_equal(dev["mi"], host["mi"])
    # an invalid window is flagged on the device and its result is NaN
    bad = w[:3].copy()
    bad["start"][1] = 29999
    dw2 = torch.from_numpy(bad.view(np.uint8)).cuda()
    dout2 = torch.zeros(3 * 40, dtype=torch.uint8, device="cuda")
    api.isycos_mi_windows_device(ctx, dw2, 3, 4, 3000, dout2, st)
    with pytest.raises(api.IsycosError):
        api.isycos_device_status(ctx, st)
    r2 = dout2.cpu().numpy().view(api.MI_OUT_DTYPE)
    assert np.isnan(r2["mi"][1]) and r2["s_psi"][0] == host["s_psi"][0]
    api.isycos_device_status(ctx, st)    # the flag was cleared


def test_invalid_arguments_are_rejected(ctx):
    api = _api()
    x = synth.normal(1, 100).astype(np.float32)
    xs = api.isycos_put_series(ctx, x)
    for starts, sizes, k in (([0], [4], 4), ([97], [5], 4), ([-1], [10], 4), ([0], [16385], 4),
                             ([0], [10], 9), ([0], [10], 0)):
        w = api.windows_array(xs, xs, starts, sizes)
        with pytest.raises(api.IsycosError) as e:
            api.isycos_mi_windows(ctx, w, k)
        assert e.value.status == api.E_INVAL
    w = api.windows_array(xs, xs + 99, [0], [10])
    with pytest.raises(api.IsycosError):
        api.isycos_mi_windows(ctx, w, 4)
    empty = api.isycos_mi_windows(ctx, api.windows_array(xs, xs, [], []), 4)
    assert empty.shape == (0,)
    bad = x.copy()
    bad[5] = np.nan
    with pytest.raises(api.IsycosError):
        api.isycos_put_series(ctx, bad)
    import torch
    bad_dev = torch.from_numpy(bad).cuda()
    bad_dev[5] = float("inf")
    with pytest.raises(api.IsycosError):
        api.isycos_put_series(ctx, bad_dev)
    api.isycos_drop_series(ctx, xs)


def test_stats_count_windows_and_pairs(ctx):
    api = _api()
    x = synth.normal(9, 1000).astype(np.float32)
    xs = api.isycos_put_series(ctx, x)
    api.isycos_reset_stats(ctx)
    w = api.windows_array(xs, xs, [0, 10, 20], [100, 200, 50])
    api.isycos_mi_windows(ctx, w, 4)
    s = api.isycos_get_stats(ctx)
    assert s["windows"] == 3 and s["pairs"] == 100 * 99 + 200 * 199 + 50 * 49
    assert s["launches"] == 1 and s["mi_kernel_launches"] == 1 and s["mi_kernel_ms"] > 0
    api.isycos_drop_series(ctx, xs)


def test_sorted_path_equals_brute_force(ctx):
    """The sub-quadratic sorted-strip path (windows of 1025..4096 points) against the
    brute-force path and the oracle, per point, on smooth, tied and degenerate data."""
    api = _api()
    n = 20000
    x, y, _ = synth.planted_pair(8, 0, n)
    base = synth.normal(synth.seed_for(204, 0), n).astype(np.float32)
    cases = [(x, y), (synth.quantize(x), synth.quantize(y)),
             (synth.quantize(x, 2.0), synth.quantize(y, 2.0)), (base, base.copy()),
             (np.full(n, 2.5, np.float32), base), (np.round(base).astype(np.float32), -base)]
    sizes = [1025, 1500, 2048, 3001, 4096]
    starts = [11, 3000, 7000, 12000, 15000]
    # windows of at most 1024 points run the sorted path in 256-thread CTAs; windows above
    # 4096 points keep its scratch in global memory
    small_sizes = [257, 300, 513, 700, 1000, 1024, 64, 100]
    small_starts = [5, 2000, 4000, 6000, 9000, 12000, 15000, 17000]
    big_sizes = [4097, 6000, 8192, 12001, 16384, 3000]
    big_starts = [0, 13000, 1000, 7000, 3000, 16000]
    for ci, (xx, yy) in enumerate(cases):
        xs, ys = api.isycos_put_series(ctx, xx), api.isycos_put_series(ctx, yy)
        for st_, sz_ in ((starts, sizes), (small_starts, small_sizes), (big_starts, big_sizes)):
            w = api.windows_array(xs, ys, st_, sz_)
            res2 = {}
            for opt in (1, 2):
                api.isycos_set_option(ctx, api.OPT_KERNEL, opt)
                res2[opt] = api.isycos_mi_windows_points(ctx, w, 4)
            api.isycos_set_option(ctx, api.OPT_KERNEL, 0)
            for a, b in zip(res2[1], res2[2]):
                assert np.array_equal(a, b), (ci, sz_)
        w = api.windows_array(xs, ys, starts, sizes)
        res = {}
        for opt in (1, 2):
            api.isycos_set_option(ctx, api.OPT_KERNEL, opt)
            res[opt] = api.isycos_mi_windows_points(ctx, w, 4)
        api.isycos_set_option(ctx, api.OPT_KERNEL, 0)
        if ci < 3:
            r = O.ksg_window(xx[3000:4500], yy[3000:4500], 4, points=False)
            assert res[2][0]["s_psi"][1] == r["s_psi"] and res[2][0]["mi"][1] == r["mi"]
        if ci == 0:   # one large window against the oracle
            api.isycos_set_option(ctx, api.OPT_KERNEL, 2)
            got = api.isycos_mi_windows(ctx, api.windows_array(xs, ys, [1000], [8192]), 4)
            api.isycos_set_option(ctx, api.OPT_KERNEL, 0)
            r = O.ksg_window(xx[1000:9192], yy[1000:9192], 4, points=False)
            assert got["s_psi"][0] == r["s_psi"] and got["mi"][0] == r["mi"]
        api.isycos_drop_series(ctx, xs)
        api.isycos_drop_series(ctx, ys)


def test_sorted_path_every_sort_form_in_one_launch(ctx):
    """One launch of 1024-thread CTAs (its largest sorted window has more than 1024 points)
    holding sorted windows whose slot counts are below, equal to, twice and four times the
    CTA's threads, and above 4096 points: the sort runs in memory, with one, two and four
    keys per thread in registers, and in global scratch.  Per-point results equal the
    brute-force path, on smooth, tied and constant data, for k = 1, 4 and 8."""
    api = _api()
    n = 30000
    x, y, _ = synth.planted_pair(8, 5, n)
    base = synth.normal(synth.seed_for(205, 0), n).astype(np.float32)
    cases = [(x, y), (synth.quantize(x), synth.quantize(y)), (np.full(n, 1.5, np.float32), base)]
    sizes = [300, 512, 513, 700, 1024, 1025, 1500, 2048, 2049, 3000, 4096, 5000, 257]
    starts = [17 + 2100 * i for i in range(len(sizes))]
    try:
        for ci, (xx, yy) in enumerate(cases):
            xs, ys = api.isycos_put_series(ctx, xx), api.isycos_put_series(ctx, yy)
            w = api.windows_array(xs, ys, starts, sizes)
            for k in (1, 4, 8):
                res = {}
                for opt in (1, 2):
                    api.isycos_set_option(ctx, api.OPT_KERNEL, opt)
                    res[opt] = api.isycos_mi_windows_points(ctx, w, k)
                for a, b in zip(res[1], res[2]):
                    assert np.array_equal(a, b), (ci, k)
            api.isycos_drop_series(ctx, xs)
            api.isycos_drop_series(ctx, ys)
    finally:
        api.isycos_set_option(ctx, api.OPT_KERNEL, 0)


def _check_points_est1(ctx, x, y, starts, sizes, k):
    api = _api()
    xs = api.isycos_put_series(ctx, x)
    ys = api.isycos_put_series(ctx, y)
    w = api.windows_array(xs, ys, starts, sizes)
    api.isycos_set_option(ctx, api.OPT_ESTIMATOR, 1)
    try:
        out, nx, ny, c = api.isycos_mi_windows_points(ctx, w, k)
        out2 = api.isycos_mi_windows(ctx, w, k)
    finally:
        api.isycos_set_option(ctx, api.OPT_ESTIMATOR, 0)
    off = 0
    for i, (s, m) in enumerate(zip(starts, sizes)):
        r = O.ksg_window(x[s:s + m], y[s:s + m], k, estimator=1)
        assert np.array_equal(nx[off:off + m], r["nx"]), (m, k, "nx")
        assert np.array_equal(ny[off:off + m], r["ny"]), (m, k, "ny")
        assert np.array_equal(c[off:off + m], r["c"]), (m, k, "c")
        assert out["s_psi"][i] == r["s_psi"] and out["s_log"][i] == r["s_log"], (m, k)
        assert abs(out["mi"][i] - r["mi"]) <= TOL and abs(out["nmi"][i] - r["nmi"]) <= TOL
        off += m
    assert np.array_equal(out2["s_psi"], out["s_psi"]) and np.array_equal(out2["mi"], out["mi"])
    api.isycos_drop_series(ctx, xs)
    api.isycos_drop_series(ctx, ys)


@pytest.mark.parametrize("k", [1, 3, 4, 8])
def test_estimator1_points_bucket_edges(ctx, k):
    """Kraskov's first estimator (strict counts in strips of half-width eps_i, psi(n + 1),
    no -1/k) on the warp path (m <= 64) and the CTA path, against the oracle per point."""
    x, y, _ = synth.planted_pair(5, k, 6000)
    sizes = [k + 1, 31, 32, 33, 64, 65, 127, 257, 700, 1024]
    starts = [(37 * i) % (6000 - 1100) for i in range(len(sizes))]
    _check_points_est1(ctx, x, y, starts, sizes, k)


@pytest.mark.parametrize("k", [3, 6])
def test_estimator1_heavy_ties(ctx, k):
    x, y, _ = synth.planted_pair(5, 10 + k, 4000)
    xq, yq = synth.quantize(x, 2.0), synth.quantize(y, 2.0)
    sizes = [20, 64, 200, 513]
    starts = [5, 300, 900, 2000]
    _check_points_est1(ctx, xq, yq, starts, sizes, k)
    dup = np.array([1, 1, 1, 1, 1, 1, 2, 2, 3], np.float32)
    _check_points_est1(ctx, dup, dup[::-1].copy(), [0], [9], 3)


def test_estimator1_sorted_plain_and_device_paths(ctx):
    """The sorted-strip path (1025..4096 points), the one-window-per-launch path and the
    device-list path give the same estimator-1 results as the brute-force path."""
    import torch
    api = _api()
    n = 12000
    x, y, _ = synth.planted_pair(8, 3, n)
    for xx, yy in ((x, y), (synth.quantize(x), synth.quantize(y))):
        xs, ys = api.isycos_put_series(ctx, xx), api.isycos_put_series(ctx, yy)
        sizes = [1025, 2048, 4096, 300]
        starts = [10, 2000, 5000, 9500]
        w = api.windows_array(xs, ys, starts, sizes)
        api.isycos_set_option(ctx, api.OPT_ESTIMATOR, 1)
        res = {}
        try:
            for opt in (1, 2):
                api.isycos_set_option(ctx, api.OPT_KERNEL, opt)
                res[opt] = api.isycos_mi_windows_points(ctx, w, 4)
            api.isycos_set_option(ctx, api.OPT_KERNEL, 0)
            plain = api.isycos_mi_windows_plain(ctx, w, 4)
            dw = torch.from_numpy(w.view(np.uint8)).cuda()
            dout = torch.empty(len(w) * 40, dtype=torch.uint8, device="cuda")
            st = torch.cuda.current_stream()
            api.isycos_mi_windows_device(ctx, dw, len(w), 4, 4096, dout, st)
            api.isycos_device_status(ctx, st)
            dev = dout.cpu().numpy().view(api.MI_OUT_DTYPE)
        finally:
            api.isycos_set_option(ctx, api.OPT_ESTIMATOR, 0)
            api.isycos_set_option(ctx, api.OPT_KERNEL, 0)
        for a, b in zip(res[1], res[2]):
            assert np.array_equal(a, b)
        assert np.array_equal(plain["s_psi"], res[1][0]["s_psi"])
        assert np.array_equal(dev["s_psi"], res[1][0]["s_psi"]) and np.array_equal(dev["mi"], res[1][0]["mi"])
        r = O.ksg_window(xx[2000:4048], yy[2000:4048], 4, points=False, estimator=1)
        assert res[2][0]["s_psi"][1] == r["s_psi"] and res[2][0]["mi"][1] == r["mi"]
        api.isycos_drop_series(ctx, xs)
        api.isycos_drop_series(ctx, ys)


def test_autotune_changes_speed_not_results(ctx):
    """isycos_autotune times the brute-force and sorted paths per eligible bucket and keeps
    the faster; every result is the same before and after, and the counters are untouched."""
    api = _api()
    n = 20000
    x, y, _ = synth.planted_pair(8, 5, n)
    xs, ys = api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)
    sizes = [100, 700, 1025, 1536, 2048, 2049, 3072, 4096, 5000]
    starts = [(997 * i) % (n - 5000) for i in range(len(sizes))]
    w = api.windows_array(xs, ys, starts, sizes)
    before = api.isycos_mi_windows(ctx, w, 4)
    st0 = api.isycos_get_stats(ctx)
    tune = api.isycos_autotune(ctx, 4)
    st1 = api.isycos_get_stats(ctx)
    assert st1["windows"] == st0["windows"] and st1["launches"] == st0["launches"]
    assert set(tune["window_size"]) == {9, 10, 11, 12, 13, 14}
    assert set(tune["sorted_buckets"]) <= {9, 10, 11, 12, 13, 14}
    assert all(v > 0 for v in tune["brute_ms"].values()) and all(v > 0 for v in tune["sorted_ms"].values())
    for b in (9, 10, 11, 12, 13, 14):
        assert (b in tune["sorted_buckets"]) == (tune["sorted_ms"][b] < tune["brute_ms"][b])
    assert tune["nt_switch"] in (512, 1024)
    if tune["sorted_buckets"]:
        b0 = min(tune["sorted_buckets"])
        if b0 <= 12:
            assert (1 << (b0 - 1)) < tune["sort_min"] <= tune["window_size"][b0]
    assert api.isycos_get_tuning(ctx, 4) == {k: tune[k] for k in ("sorted_buckets", "sort_min", "nt_switch")}
    after = api.isycos_mi_windows(ctx, w, 4)
    assert np.array_equal(before, after)
    api.isycos_drop_series(ctx, xs)
    api.isycos_drop_series(ctx, ys)


def test_ring_shaped_batch_all_paths_agree(ctx):
    """2,000 windows of 32..1024 points (log-uniform, the shape of BU rings): the plain
    one-window-per-launch form, the brute-force batch and the sorted-path batch give the same
    integers, and sampled windows equal the oracle."""
    api = _api()
    n = 100000
    x, y, _ = synth.planted_pair(2, 0, n)
    xs, ys = api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)
    rng = np.random.default_rng(5)
    sizes = np.exp(rng.uniform(np.log(32), np.log(1024), 2000)).astype(int)
    starts = np.array([int(rng.integers(0, n - m)) for m in sizes])
    w = api.windows_array(xs, ys, starts, sizes)
    res = {}
    try:
        for opt in (1, 2):
            api.isycos_set_option(ctx, api.OPT_KERNEL, opt)
            res[opt] = api.isycos_mi_windows(ctx, w, 4)
    finally:
        api.isycos_set_option(ctx, api.OPT_KERNEL, 0)
    plain = api.isycos_mi_windows_plain(ctx, w, 4)
    bad = np.nonzero(res[1]["s_psi"] != res[2]["s_psi"])[0]
    assert bad.size == 0, ("sorted vs brute", bad[:10], sizes[bad[:10]])
    bad = np.nonzero(plain["s_psi"] != res[1]["s_psi"])[0]
    assert bad.size == 0, ("plain vs brute", bad[:10], sizes[bad[:10]])
    for i in range(0, 2000, 97):
        s, m = int(starts[i]), int(sizes[i])
        r = O.ksg_window(x[s:s + m], y[s:s + m], 4, points=False)
        assert res[1]["s_psi"][i] == r["s_psi"] and res[1]["mi"][i] == r["mi"], (i, m)
    api.isycos_drop_series(ctx, xs)
    api.isycos_drop_series(ctx, ys)


def test_sorted_path_y_order_points(ctx):
    """Above 1,024 points the sorted path sends a point whose y neighbourhood is sparse (far
    from the others in y) to a second scan along the y order.  Heavy-tailed y values (a
    ratio of normals), coarse ties in y among those outliers, ties in x, and heavy tails in
    both coordinates make many points take it; per point the results equal the brute-force
    path for k = 1, 4 and 8, and one window per case equals the oracle."""
    api = _api()
    n = 40000
    a = synth.normal(synth.seed_for(206, 0), n)
    b = synth.normal(synth.seed_for(206, 1), n)
    c = synth.normal(synth.seed_for(206, 2), n)
    heavy = (b / np.where(np.abs(c) < 1e-3, 1e-3, c)).astype(np.float32)   # Cauchy-like tails
    x = a.astype(np.float32)
    cases = [(x, heavy), (x, synth.quantize(heavy, 0.5)), (synth.quantize(x, 4.0), heavy),
             ((a / np.where(np.abs(b) < 1e-3, 1e-3, b)).astype(np.float32), heavy)]
    sizes = [1025, 1800, 2048, 3333, 4096, 4097, 7000, 16384]
    starts = [100 + 2900 * i for i in range(len(sizes))]
    try:
        for ci, (xx, yy) in enumerate(cases):
            xs, ys = api.isycos_put_series(ctx, xx), api.isycos_put_series(ctx, yy)
            w = api.windows_array(xs, ys, starts, sizes)
            for k in (1, 4, 8):
                res = {}
                for opt in (1, 2):
                    api.isycos_set_option(ctx, api.OPT_KERNEL, opt)
                    res[opt] = api.isycos_mi_windows_points(ctx, w, k)
                for u, v in zip(res[1], res[2]):
                    assert np.array_equal(u, v), (ci, k)
            s0, m0 = starts[1], sizes[1]
            r = O.ksg_window(xx[s0:s0 + m0], yy[s0:s0 + m0], 4, points=False)
            api.isycos_set_option(ctx, api.OPT_KERNEL, 2)
            got = api.isycos_mi_windows(ctx, api.windows_array(xs, ys, [s0], [m0]), 4)
            assert got["s_psi"][0] == r["s_psi"] and got["s_log"][0] == r["s_log"], ci
            api.isycos_drop_series(ctx, xs)
            api.isycos_drop_series(ctx, ys)
    finally:
        api.isycos_set_option(ctx, api.OPT_KERNEL, 0)


def test_sorted_path_repeats_bit_exact(ctx):
    """The sorted path's sorts and scans synchronise warps and CTAs in many small steps; a
    missing barrier shows up as run-to-run differences.  Repeat mixed batches (256- and
    1024-thread CTAs) and require every repeat to equal the brute-force path."""
    api = _api()
    n = 60000
    x, y, _ = synth.planted_pair(2, 7, n)
    xs, ys = api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)
    rng = np.random.default_rng(11)
    lists = []
    for lo, hi, cnt in ((257, 1024, 600), (1025, 4096, 600), (4097, 16384, 40)):
        sizes = rng.integers(lo, hi + 1, cnt)
        starts = np.array([int(rng.integers(0, n - m)) for m in sizes])
        lists.append(api.windows_array(xs, ys, starts, sizes))
    try:
        for w in lists:
            api.isycos_set_option(ctx, api.OPT_KERNEL, 1)
            ref = api.isycos_mi_windows(ctx, w, 4)
            api.isycos_set_option(ctx, api.OPT_KERNEL, 2)
            for rep in range(12):
                got = api.isycos_mi_windows(ctx, w, 4)
                bad = np.nonzero(got["s_psi"] != ref["s_psi"])[0]
                assert bad.size == 0, (rep, bad[:8], w["m"][bad[:8]])
    finally:
        api.isycos_set_option(ctx, api.OPT_KERNEL, 0)
    api.isycos_drop_series(ctx, xs)
    api.isycos_drop_series(ctx, ys)


def _sort_cx(m):
    lg = 0
    while (1 << lg) < m:
        lg += 1
    return (1 << lg) * lg * (lg + 1) // 2


def test_work_counters_follow_the_path_taken(ctx):
    """The statistics count the work each path really does: m x m point x candidate
    evaluations per brute-force window; per sorted-path window the compare-exchange steps of
    its two bitonic sorts (closed form), at least the 48..64 points around every point in the
    outward scans, and binary-search steps (about five searches of log2 m steps per point)."""
    api = _api()
    n = 30000
    x, y, _ = synth.planted_pair(2, 11, n)
    xs, ys = api.isycos_put_series(ctx, x), api.isycos_put_series(ctx, y)
    sizes = [40, 100, 300, 1025, 2048, 4096]
    starts = [100 + 4500 * i for i in range(len(sizes))]
    w = api.windows_array(xs, ys, starts, sizes)
    try:
        api.isycos_set_option(ctx, api.OPT_KERNEL, 1)
        api.isycos_reset_stats(ctx)
        r1 = api.isycos_mi_windows(ctx, w, 4)
        st = api.isycos_get_stats(ctx)
        assert st["work_bf"] == sum(m * m for m in sizes)
        assert st["work_scan"] == st["work_search"] == st["work_sort"] == 0
        api.isycos_set_option(ctx, api.OPT_KERNEL, 2)
        api.isycos_reset_stats(ctx)
        r2 = api.isycos_mi_windows(ctx, w, 4)
        st = api.isycos_get_stats(ctx)
    finally:
        api.isycos_set_option(ctx, api.OPT_KERNEL, 0)
    assert np.array_equal(r1, r2)
    # the launch runs 1024-thread CTAs (its largest sorted window has more than 1024 points):
    # windows of 257..512 points then run two per CTA, by brute force
    big = [m for m in sizes if m > 512]
    assert st["work_bf"] == sum(m * m for m in sizes if m <= 512)
    assert st["work_sort"] == sum(_sort_cx(m) for m in big)
    assert st["work_scan"] >= sum(m * 48 for m in big)
    assert st["work_scan"] < sum(m * m for m in big)
    lg = {m: int(np.ceil(np.log2(m))) for m in big}
    assert sum(3 * m * (lg[m] - 2) for m in big) <= st["work_search"] <= sum(6 * m * (lg[m] + 1) for m in big)
    api.isycos_drop_series(ctx, xs)
    api.isycos_drop_series(ctx, ys)


def test_put_series_many_and_reuse_of_dropped_memory(ctx):
    """isycos_put_series_many makes several series resident with one synchronisation; a
    batch holding a non-finite value makes none resident; dropped series leave their memory
    to the next series of about their size, so a put / drop cycle allocates nothing."""
    import torch
    api = _api()
    n = 50000
    pairs = [synth.planted_pair(2, 20 + p, n)[:2] for p in range(4)]
    flat = api.isycos_put_series_many(ctx, [a for xy in pairs for a in xy])
    assert len(set(flat)) == 8
    w = api.windows_array(flat[0], flat[1], [0, 1000, 30000], [64, 700, 4096])
    ref = api.isycos_mi_windows(ctx, w, 4)
    bad = [pairs[0][0].copy(), pairs[0][1].copy()]
    bad[1][17] = np.inf
    with pytest.raises(api.IsycosError) as e:
        api.isycos_put_series_many(ctx, bad)
    assert e.value.status == api.E_INVAL
    for sid in flat:
        api.isycos_drop_series(ctx, sid)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for rep in range(3):   # the same sizes again: the kept buffers serve them
        dev = [torch.from_numpy(a).cuda() for xy in pairs for a in xy]
        torch.cuda.synchronize()
        free_t, _ = torch.cuda.mem_get_info()
        ids = api.isycos_put_series_many(ctx, dev)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free_t, (rep, free_t, free1)
        got = api.isycos_mi_windows(ctx, api.windows_array(ids[0], ids[1], [0, 1000, 30000], [64, 700, 4096]), 4)
        assert np.array_equal(got, ref)
        for sid in ids:
            api.isycos_drop_series(ctx, sid)
        del dev


def test_tuning_file_is_written_and_loaded(tmp_path, monkeypatch):
    """isycos_autotune stores its choice under the GPU's name and k in ISYCOS_TUNING_FILE; a
    context created later loads it (and a line for another GPU is left alone)."""
    api = _api()
    path = tmp_path / "tuning.json"
    path.write_text('{"gpu": "another GPU", "k": 4, "sorted_buckets": 512, "sort_min": 300, "nt_switch": 512}\n')
    monkeypatch.setenv("ISYCOS_TUNING_FILE", str(path))
    with api.Context(0) as c1:
        assert api.isycos_get_tuning(c1, 3) is None
        tune = api.isycos_autotune(c1, 3)
        got = api.isycos_get_tuning(c1, 3)
    lines = path.read_text().splitlines()
    assert len(lines) == 2 and "another GPU" in lines[0] and '"k": 3' in lines[1]
    with api.Context(0) as c2:
        assert api.isycos_get_tuning(c2, 3) == got
        assert api.isycos_get_tuning(c2, 4) is None
    assert got["sort_min"] == tune["sort_min"] and got["nt_switch"] == tune["nt_switch"]
