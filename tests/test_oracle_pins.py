"""The oracle against what the paper and the mathematics fix (no GPU)."""
import pytest

import oracle_pins as P


@pytest.mark.parametrize("pin", P.PINS, ids=[p.__name__ for p in P.PINS])
def test_pin(pin):
    ok, detail = pin()
    assert ok, detail
