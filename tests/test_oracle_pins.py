"""The CPU oracle against what the paper and the mathematics fix (no GPU)."""
import pytest

import oracle_pins as P


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    fails = pin()
    assert not fails, "\n".join(fails)
