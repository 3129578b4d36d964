"""The oracle against closed forms, brute force and invariants (CPU only)."""
import pytest

import oracle

from tests.oracle_pins import ALL_PINS


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(oracle.load())
