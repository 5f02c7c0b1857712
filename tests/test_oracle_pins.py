"""The oracle against what the paper and mathematics fix (CPU only)."""
import pytest

import oracle
from oracle_pins import ALL_PINS, pin_lower_bound_exhaustive


@pytest.fixture(scope="module")
def O():
    return oracle.get()


@pytest.mark.parametrize("pin", [p for p in ALL_PINS
                                 if p is not pin_lower_bound_exhaustive],
                         ids=lambda p: p.__name__)
def test_pin(O, pin):
    pin(O)


def test_lower_bound_exhaustive_m_le_5(O):
    """Every ACGT pair of length 1..5, E = 0..3: no pair within E edits is
    rejected and the count never exceeds the edit distance (Theorem 2)."""
    pin_lower_bound_exhaustive(O, mmax=5, Emax=3)


def test_default_threads_positive(O):
    assert O.default_threads() >= 1
