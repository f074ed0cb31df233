"""Planted mistakes in the oracle (CPU only): each must fail at least one pin.

The oracle carries a switch that re-introduces one plausible mistake at a time.  In the
estimator: a dropped term, a strict instead of inclusive count, the point counted as its own
neighbour, Kraskov's first estimator, a swapped dimension, the other tie-break, the
Euclidean norm, the garbled entropy sign, psi(m - 1).  In the searches: acceptance with >=,
the last maximum of a ring winning, no s_min floor on the TD layer size, an extension window
w_delta that overlaps w_o, Def. 6.2 without its I > 0 condition, the whole square instead of
the ring N_r, a noisy side dropping both sides, plain hill climbing without the
late-acceptance history, chunks without their s_max overlap, and a selection runtime that
counts windows instead of pair comparisons, a noise test on extensions of fewer than
k + 1 points, a detection count that is not reset by a TD window or a BU step that is
not noise, a TD layer that also scores (and keeps) a window ending at its partition's end,
and a selection sample drawn from the generator's outputs 0 .. m-1 instead of 1 .. m.  With
the switch on, the pins of
``tests/_pins.py`` and ``tests/_search_pins.py`` must notice.
"""
import pytest

from oracle import oracle as O
from tests import _pins, _search_pins


def _failures():
    failed = []
    for pin in _pins.FAST_PINS + _search_pins.SEARCH_PINS:
        try:
            pin()
        except AssertionError:
            failed.append(pin.__name__)
    return failed


def test_no_mutation_passes_all_pins():
    assert _failures() == []


@pytest.mark.parametrize("name", [n for n in O.MUTATIONS if n != "none"])
def test_mutation_is_caught(name):
    with O.mutation(name):
        failed = _failures()
    assert failed, "planted mistake %r passed every pin" % name
