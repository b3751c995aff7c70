"""The CPU oracle against facts fixed by the definitions (Sec. 3.1) and by
mathematics: closed forms, exact integer sums, exact rational brute force and
invariants.  See tests/pins.py for the list."""
import pytest

import oracle
import pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(oracle.Oracle())
