"""gm_cardinality's sum on adversarial register values (GPU), against the
correctly rounded sum of Python's math.fsum: the estimate (k - 1) / sum y must
agree within k 2^-52 relative (the documented bound of an FP64 sum of k
non-negative terms in any order), and the same row must give the same bits on
every call."""
import math

import numpy as np
import pytest
import torch

from paper_2302_05176_gb300 import gm

pytestmark = pytest.mark.gpu


def _fsum_card(y):
    return [(row.size - 1) / math.fsum(row.tolist()) if np.all(np.isfinite(row)) else 0.0 for row in y]


@pytest.mark.parametrize("k", [2, 3, 31, 64, 1023, 1024, 4096])
def test_cardinality_sum_is_correctly_rounded(k):
    rng = np.random.default_rng(k)
    rows = [
        rng.exponential(size=k),                                   # a sketch's registers
        np.exp(rng.uniform(-40, 40, size=k)),                      # 115 binades of dynamic range
        np.full(k, 1.0) + rng.integers(0, 2, k) * 2.0 ** -52,      # sums with rounding ties
        np.exp(rng.uniform(-700, -690, size=k)),                   # tiny values
        np.concatenate([[5e-324, 1e-310], np.full(k - 2, 1e-300)]) if k > 2 else np.array([5e-324, 1e-310]),
        np.concatenate([[0.0], rng.exponential(size=k - 1)]),      # a zero register (an underflowed arrival)
        np.full(k, 2.0 ** 1000),                                   # large values
    ]
    y = np.stack(rows).astype(np.float64)
    want = _fsum_card(y)
    got = gm.gm_cardinality(torch.from_numpy(y).cuda()).cpu().numpy()
    for r in range(y.shape[0]):
        assert got[r] == pytest.approx(want[r], rel=k * 2.0 ** -52, abs=0), (k, r, got[r], want[r])
    again = gm.gm_cardinality(torch.from_numpy(y).cuda()).cpu().numpy()
    assert np.array_equal(again.view(np.int64), got.view(np.int64))
    # an unfilled register estimates 0; a misaligned row (odd offset) takes the scalar path
    y2 = y.copy()
    y2[0, k // 2] = np.inf
    assert gm.gm_cardinality(torch.from_numpy(y2).cuda()).cpu().numpy()[0] == 0.0
    if k % 2 == 0:
        flat = torch.from_numpy(np.concatenate([[0.0], y[1]])).cuda()
        one = gm.gm_cardinality(flat[1:].view(1, k)).cpu().numpy()[0]
        assert one == pytest.approx(want[1], rel=k * 2.0 ** -52, abs=0)
