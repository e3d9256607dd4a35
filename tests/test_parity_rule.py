"""The GPU-vs-oracle comparison rule itself (CPU only): planted differences in a
copy of an oracle sketch must fail it, allowed ones must pass."""
import numpy as np

import oracle
from paper_2302_05176_gb300 import workloads as W
from parity import compare_sketch


def _ulps(x, n):
    return (np.asarray(x, np.float64).view(np.int64) + n).view(np.float64)


def _case():
    X = W.lognormal_batch(seed=3, n_rows=6, median=200.0, hi=600)
    s, y, y2, s2 = oracle.sketch(X.row_ptr, X.ids, X.w, 64, 5, runner_up=True)
    return s, y, y2, s2


def test_identical_and_within_four_ulp_pass():
    s, y, y2, s2 = _case()
    assert compare_sketch(s, y, s, y, y2, s2)["ok"]
    rep = compare_sketch(s, _ulps(y, 4), s, y, y2, s2)
    assert rep["ok"] and rep["max_ulp"] == 4


def test_five_ulp_fails_everywhere():
    s, y, y2, s2 = _case()
    for n in (5, -5):
        yb = y.copy()
        yb[2, 7] = _ulps(y[2, 7], n)
        assert not compare_sketch(s, yb, s, y, y2, s2)["ok"]


def test_near_tie_rules():
    s, y, y2, s2 = _case()
    # make register (1, 3) a near-tie: the runner-up 1e-13 relative above the winner
    y2t, s2t = y2.copy(), s2.copy()
    y2t[1, 3] = y[1, 3] * (1 + 1e-13)
    s2t[1, 3] = s[1, 3] + 1
    # the GPU took the runner-up: allowed when its value is the runner-up's time
    sg, yg = s.copy(), y.copy()
    sg[1, 3], yg[1, 3] = s2t[1, 3], y2t[1, 3]
    rep = compare_sketch(sg, yg, s, y, y2t, s2t)
    assert rep["ok"] and rep["tie_index_flips"] == 1
    # ... but not with the winner's value (hundreds of ulp from the runner-up's)
    yg2 = yg.copy()
    yg2[1, 3] = y[1, 3]
    assert not compare_sketch(sg, yg2, s, y, y2t, s2t)["ok"]
    # a same-id near-tie register is held to 4 ulp too
    yg3 = y.copy()
    yg3[1, 3] = _ulps(y[1, 3], 9)
    assert not compare_sketch(s, yg3, s, y, y2t, s2t)["ok"]
    # an id that is neither the winner nor the runner-up fails
    sg4 = s.copy()
    sg4[1, 3] = s[1, 3] + 2
    assert not compare_sketch(sg4, y, s, y, y2t, s2t)["ok"]
    # without the near-tie, taking the runner-up fails
    assert not compare_sketch(sg, yg, s, y, y2, s2)["ok"] or y2[1, 3] - y[1, 3] <= 1e-12 * y[1, 3]


def test_filled_pattern_and_unfilled_ids():
    s, y, y2, s2 = _case()
    yb, sb = y.copy(), s.copy()
    yb[0, 0], sb[0, 0] = np.inf, -1
    assert not compare_sketch(sb, yb, s, y, y2, s2)["ok"]
    rows = [(np.array([4, 5], np.int32), np.array([0.0, 0.0]))]
    Z = W.from_rows(rows)
    sz, yz, y2z, s2z = oracle.sketch(Z.row_ptr, Z.ids, Z.w, 8, 1, runner_up=True)
    assert np.all(sz == -1) and np.all(s2z == -1) and np.all(np.isinf(y2z))
    assert compare_sketch(sz, yz, sz, yz, y2z, s2z)["ok"]
    sz2 = sz.copy()
    sz2[0, 1] = 4
    assert not compare_sketch(sz2, yz, sz, yz, y2z, s2z)["ok"]
