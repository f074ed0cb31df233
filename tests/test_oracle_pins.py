"""The CPU oracle against the facts the paper and the mathematics fix (no GPU)."""
import math

import numpy as np
import pytest
from scipy.special import digamma

from oracle import oracle as O
from paper_2204_09131_gb300 import synth
from tests import _pins


def test_digamma_table_matches_scipy():
    psi = O.digamma_table(70000)
    n = np.arange(1, 70001)
    ref = digamma(n.astype(np.float64))
    assert np.max(np.abs(psi[1:] - ref)) < 1e-11
    assert psi[1] == pytest.approx(-0.5772156649015329, abs=1e-16)


def test_fixed_tables_round_scipy_values():
    psi_fx, log_fx = O.fixed_tables(40000)
    n = np.arange(1, 40001)
    ref = np.rint(np.ldexp(digamma(n.astype(np.float64)), 32)).astype(np.int64)
    diff = np.abs(psi_fx[1:] - ref)
    assert diff.max() <= 1 and np.mean(diff == 0) > 0.999
    ref_log = np.rint(np.ldexp(np.log(n.astype(np.float64)), 32)).astype(np.int64)
    assert np.array_equal(log_fx[1:], ref_log)
    assert psi_fx[0] == 0 and log_fx[0] == 0


@pytest.mark.parametrize("pin", _pins.FAST_PINS, ids=lambda f: f.__name__)
def test_fast_pin(pin):
    pin()


@pytest.mark.parametrize("estimator", [0, 1])
def test_gaussian_closed_form_and_independence(estimator):
    _pins.pin_gaussian(estimator=estimator)


def test_gaussian_large_window():
    # m = 1024, rho = 0.8: -1/2 ln(1 - 0.64) = 0.5108
    vals = []
    for w in range(8):
        x, y = synth.gaussian_pair(synth.seed_for(95, 0, w), 1024, 0.8)
        vals.append(O.ksg_window(x, y, 4, points=False)["mi_exact"])
    vals = np.array(vals)
    se = vals.std(ddof=1) / math.sqrt(len(vals))
    assert abs(vals.mean() - (-0.5 * math.log(1 - 0.64))) < 4 * se + 0.02


def test_monotone_transform_within_estimator_error():
    # Max-norm kNN is not rank based, so invariance holds in expectation only.
    a, b, c = [], [], []
    for w in range(12):
        x, y = synth.gaussian_pair(synth.seed_for(96, 0, w), 256, 0.7)
        a.append(O.ksg_window(x, y, 4, points=False)["mi_exact"])
        b.append(O.ksg_window(np.exp(x).astype(np.float32), y, 4, points=False)["mi_exact"])
        c.append(O.ksg_window(x ** 3, y, 4, points=False)["mi_exact"])
    a, b, c = map(np.mean, (a, b, c))
    assert abs(a - b) < 0.08 and abs(a - c) < 0.08, (a, b, c)


def test_point_function_matches_window_function():
    x, y = synth.gaussian_pair(synth.seed_for(97, 0), 150, 0.4)
    r = O.ksg_window(x, y, 4)
    for i in (0, 1, 77, 149):
        p = O.ksg_point(x, y, 4, i)
        assert (p["nx"], p["ny"], p["c"]) == (r["nx"][i], r["ny"][i], r["c"][i])
        assert np.float32(p["eps"]) == r["eps"][i]


def test_counts_bounds():
    # Every point has at least k neighbours inside both strips; c_i >= 1.
    x, y = synth.gaussian_pair(synth.seed_for(98, 0), 300, 0.2)
    for xx, yy in ((x, y), (synth.quantize(x, 2.0), synth.quantize(y, 2.0))):
        r = O.ksg_window(xx, yy, 5)
        assert r["nx"].min() >= 5 and r["ny"].min() >= 5 and r["c"].min() >= 1
        assert r["nx"].max() <= 299 and r["ny"].max() <= 299


def test_invalid_sizes_rejected():
    x = np.zeros(4, np.float32)
    with pytest.raises(ValueError):
        O.ksg_window(x, x, 4)          # m < k + 1


def test_splitmix64_reference_values():
    # SplitMix64 with state 1234567 (Vigna's splitmix64.c): first outputs of the stream.
    assert O.splitmix64_at(1234567, 1) == 6457827717110365317
    assert O.splitmix64_at(1234567, 2) == 3203168211198807973
    vals = synth.splitmix64(1234567, 2)
    assert int(vals[0]) == 6457827717110365317 and int(vals[1]) == 3203168211198807973
