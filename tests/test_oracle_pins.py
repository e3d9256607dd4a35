"""The CPU oracle against what the paper and the mathematics fix (no GPU)."""
import numpy as np
import pytest

import oracle
import oracle_pins as P


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    fails = pin()
    assert not fails, "\n".join(fails)


def test_fastsearch_phase_by_brute_force():
    """Algorithm 1's FastSearch phase (the budget R at which every server is first
    filled, and the arrivals released by then) recomputed from each element's full
    arrival list: release the first min(k, ceil(R v_i / sum v)) arrivals of every
    element for R = delta, 2 delta, ... until the released arrivals cover all k
    servers."""
    import math
    rng = np.random.default_rng(77)
    for k, n, delta in ((16, 40, 16), (32, 12, 5), (8, 300, 8)):
        ids = rng.choice(1 << 20, n, replace=False).astype(np.int32)
        w = rng.exponential(size=n)
        _, _, _, R_alg, arr_alg = oracle.fastgm_alg1(ids, w, k, 3, delta=delta, search=True)
        lists = [oracle.arrivals(int(i), float(v), k, 3)[1] for i, v in zip(ids, w)]
        total = float(np.sum(w))
        R = 0
        while True:
            R += delta
            lens = [min(k, math.ceil(R * (v / total))) for v in w]
            covered = set()
            for c, m in zip(lists, lens):
                covered.update(int(x) for x in c[:m])
            if len(covered) == k:
                break
        assert R == R_alg and sum(lens) == arr_alg, (k, n, R, R_alg, sum(lens), arr_alg)
