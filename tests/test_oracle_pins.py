"""The CPU oracle against independent pins (Floyd-Warshall, closed forms,
hand-derived lists, polynomial roots; closed-form eigenvectors for the
spectral layout). CPU only."""
import pytest

import oracle
import oracle_pins as pins
import spectral_pins as spins
from oracle import spectral


@pytest.fixture(scope="module")
def orc():
    return oracle.default()


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda c: c.__name__)
def test_pin(orc, check):
    check(orc)


@pytest.mark.parametrize("check", spins.ALL_CHECKS, ids=lambda c: c.__name__)
def test_spectral_pin(check):
    check(spectral)
