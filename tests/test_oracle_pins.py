"""The CPU oracle against independent pins (Floyd-Warshall, closed forms,
hand-derived lists, polynomial roots). CPU only."""
import pytest

import oracle
import oracle_pins as pins


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda c: c.__name__)
def test_pin(orc, check):
    check(orc)
