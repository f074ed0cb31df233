"""Planted mistakes in the oracle (CPU only): each must fail at least one pin.

The oracle carries a switch that re-introduces one plausible mistake at a time (a dropped
term, a strict instead of inclusive count, the point counted as its own neighbour,
Kraskov's first estimator, a swapped dimension, the other tie-break, the Euclidean norm,
the garbled entropy sign, psi(m - 1)).  With the switch on, the pins of
``tests/_pins.py`` must notice.
"""
import pytest

from oracle import oracle as O
from tests import _pins


def _failures():
    failed = []
    for pin in _pins.FAST_PINS:
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
