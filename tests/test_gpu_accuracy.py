"""Accuracy of the GPU sketches against the paper's theory (Sec. 2.4): the
Jaccard estimate is unbiased with Var = J_P (1 - J_P) / k, and the cardinality
estimate (k - 1) / sum y has relative variance 1 / (k - 2).  Seeds are fixed;
the bands are about 4 standard errors of an RMSE estimated from the replicate
count."""
import math

import numpy as np
import pytest

from paper_2302_05176_gb300 import accuracy

pytestmark = pytest.mark.gpu


def test_probability_jaccard_definition():
    # identical vectors: 1; disjoint: 0; u = 2v on the same ids: 1 (scale-free)
    ids = np.array([3, 7, 9])
    w = np.array([0.5, 1.0, 2.0])
    assert accuracy.probability_jaccard(ids, w, ids, w) == pytest.approx(1.0)
    assert accuracy.probability_jaccard(ids, w, ids + 100, w) == 0.0
    assert accuracy.probability_jaccard(ids, w, ids, 2 * w) == pytest.approx(1.0)
    # a hand case: u = (1, 1), v = (1, 0): J_P = 1 / (max(1,1) + max(1,0)) = 1/2
    assert accuracy.probability_jaccard(np.array([1, 2]), np.array([1.0, 1.0]), np.array([1]),
                                        np.array([1.0])) == pytest.approx(0.5)


def test_jaccard_rmse_matches_theory():
    res = accuracy.jaccard_rmse(ks=(64, 256, 1024), n_pairs=30, n_pos=400, reps=48)
    m = res["pairs"] * res["replications"]
    for row in res["by_k"]:
        band = 4.0 / math.sqrt(2 * m)  # relative standard error of an RMSE from m squared errors
        assert abs(row["rmse"] / row["theory"] - 1) < band + 0.05, row
        assert abs(row["bias"]) < 4 * row["theory"] / math.sqrt(m), row


def test_cardinality_rmse_matches_theory():
    res = accuracy.cardinality_rmse(ks=(64, 256, 1024), ns=(100, 3000), reps=120)
    for row in res["rows"]:
        assert abs(row["rel_rmse"] / row["theory"] - 1) < 4.0 / math.sqrt(2 * 120) + 0.05, row
        assert abs(row["bias"]) < 4 * row["theory"] / math.sqrt(120) + 1.0 / (row["k"] - 2), row
