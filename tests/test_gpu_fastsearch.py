"""The paper's FastSearch schedule on the GPU (gm_sketch_fastsearch, gm_sketch_budget,
gm_sketch_bounded): its rounds and released arrivals equal the oracle's Algorithm 1
when the row sums are exact in any order (dyadic weights), and FastSearch +
FastPrune give gm_sketch's registers; caller-given bounds of any value give them
too."""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_05176_gb300 import fastsearch, gm
from paper_2302_05176_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def dyadic_rows(seed, lens):
    """Weights m 2^-12 with m < 2^20: every partial sum is exact, so a row's FP64
    sum is the same in any order."""
    rng = np.random.default_rng(seed)
    rows = []
    for n in lens:
        ids = rng.choice(1 << 24, n, replace=False).astype(np.int32)
        m = np.maximum(1, np.floor(rng.exponential(size=n) * 2 ** 10)).astype(np.float64)
        rows.append((ids, m * 2.0 ** -12))
    return W.from_rows(rows)


@pytest.mark.parametrize("k,delta", [(16, 16), (64, 64), (256, 100)])
def test_fastsearch_matches_algorithm_1(k, delta):
    """The device schedule (gm_sketch_fastsearch) takes, for every row, the rounds
    Algorithm 1 takes, and gives gm_sketch's registers; the budgets of its last
    round release the arrivals Algorithm 1's FastSearch released."""
    X = dyadic_rows(k, [1, 3, 40, 200, 900, 40000])  # the last one longer than a chunk
    rp, ids, w = gm.to_device(X)
    s, y, info = fastsearch.fastsearch_sketch(rp, ids, w, k, 7, delta=delta)
    s0, y0, _ = gm.gm_sketch(rp, ids, w, k, 7)
    assert torch.equal(s, s0) and torch.equal(y.view(torch.int64), y0.view(torch.int64))
    rounds = info["rounds"].cpu().numpy()
    R_dev = torch.zeros(X.n_rows, dtype=torch.float64, device="cuda")
    total = 0
    for r in range(X.n_rows):
        lo, hi = X.row_ptr[r], X.row_ptr[r + 1]
        _, _, _, R_alg, arr_alg = oracle.fastgm_alg1(X.ids[lo:hi], X.w[lo:hi], k, 7, delta=delta, search=True)
        assert rounds[r] * delta == R_alg, (r, rounds[r], R_alg)
        R_dev[r] = float(R_alg)
        total += arr_alg
    # the release step alone at those budgets (gm_sketch_budget) fills every register
    # with the arrivals Algorithm 1 released
    sb, yb, wsb = gm.gm_sketch_budget(rp, ids, w, k, 7, R_dev)
    assert gm.gm_status(wsb)[1]["arrivals"] == total
    assert bool(torch.isfinite(yb).all())


def test_fastsearch_wide_shape_k4096():
    """k = 4096 runs the schedule on 1024-thread CTAs: rounds equal Algorithm 1's,
    registers equal gm_sketch's, on dyadic rows including one of 40,000 elements."""
    k, delta = 4096, 4096
    X = dyadic_rows(99, [2, 50, 700, 3000, 40000])
    rp, ids, w = gm.to_device(X)
    s, y, info = fastsearch.fastsearch_sketch(rp, ids, w, k, 11, delta=delta)
    s0, y0, _ = gm.gm_sketch(rp, ids, w, k, 11)
    assert torch.equal(s, s0) and torch.equal(y.view(torch.int64), y0.view(torch.int64))
    rounds = info["rounds"].cpu().numpy()
    for r in range(X.n_rows):
        lo, hi = X.row_ptr[r], X.row_ptr[r + 1]
        _, _, _, R_alg, _ = oracle.fastgm_alg1(X.ids[lo:hi], X.w[lo:hi], k, 11, delta=delta, search=True)
        assert rounds[r] * delta == R_alg, (r, rounds[r], R_alg)


def test_fastsearch_on_lognormal_rows():
    """Non-dyadic weights, k = 1024: the same registers as gm_sketch, rounds > 1."""
    X = W.lognormal_batch(seed=31, n_rows=48, median=1500.0, hi=40000)
    rp, ids, w = gm.to_device(X)
    s, y, info = fastsearch.fastsearch_sketch(rp, ids, w, 1024, 5)
    s0, y0, _ = gm.gm_sketch(rp, ids, w, 1024, 5)
    assert torch.equal(s, s0) and torch.equal(y.view(torch.int64), y0.view(torch.int64))
    assert info["max_rounds"] > 1 and bool((info["rounds"] >= 1).all())


def test_bounds_of_any_value_give_the_same_registers():
    X = W.lognormal_batch(seed=21, n_rows=64, median=800.0)
    rp, ids, w = gm.to_device(X)
    k = 512
    s0, y0, _ = gm.gm_sketch(rp, ids, w, k, 3)
    ystar = gm.gm_row_ystar(y0)
    for b in (ystar, ystar * 0.5, ystar * 1e-6, ystar * 1e6, torch.full_like(ystar, float("inf")),
              torch.full_like(ystar, float("nan")), torch.full_like(ystar, -1.0), torch.full_like(ystar, 1e-300)):
        s, y, _ = gm.gm_sketch_bounded(rp, ids, w, k, 3, b.contiguous())
        assert torch.equal(s, s0) and torch.equal(y.view(torch.int64), y0.view(torch.int64))
    # y* itself as the bound: no row needs a second pass
    _, _, ws = gm.gm_sketch_bounded(rp, ids, w, k, 3, ystar)
    assert gm.gm_status(ws)[1]["rows_fallback"] == 0


def test_row_ystar():
    y = torch.tensor([[1.0, 3.0, 2.0], [5.0, float("inf"), 0.5]], dtype=torch.float64, device="cuda")
    assert gm.gm_row_ystar(y).tolist() == [3.0, float("inf")]
