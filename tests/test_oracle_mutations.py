"""Planted mistakes in the oracle (CPU only): each must trip at least one pin.

Mutations (set inside the C oracle through gmo_set_mutation):
  1  divisor 1/k instead of 1/(k-z): arrivals are no longer order statistics
  2  divisor 1/(k-z+1) with the 0-based step: off by one
  3  no Fisher-Yates shuffle: servers visited in order
  4  server read from the wrong slot after the swap
  5  uniform built from the wrong bits
  6  register ties go to the larger id
"""
import pytest

import oracle
import oracle_pins as P

CHECKS = {
    1: [P.pin_order_statistics],
    2: [P.pin_order_statistics],
    3: [P.pin_server_uniformity],
    4: [P.pin_server_uniformity],
    5: [P.pin_order_statistics, P.pin_uniform_and_randint],
    6: [P.pin_merge_and_scale],
}


@pytest.mark.parametrize("mutation", sorted(CHECKS))
def test_planted_mistake_is_caught(mutation):
    with oracle.mutation(mutation):
        fails = [msg for pin in CHECKS[mutation] for msg in pin()]
    assert fails, "mutation %d passed every pin" % mutation
    # and the unmutated oracle passes the same pins
    assert not [msg for pin in CHECKS[mutation] for msg in pin()]
