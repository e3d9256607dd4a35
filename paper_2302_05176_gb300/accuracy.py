"""Accuracy of the GPU sketches: the paper's synthetic accuracy experiments
(Task 1: probability-Jaccard RMSE against k; Task 2: weighted-cardinality RMSE
against n and k, weights UNI(0,1) and N(1, 0.1)) replicated on synthetic inputs.

Replications: the arrivals of an element depend on (seed, id), so shifting every
id of an input by r 2^24 gives an independent replication of the same weighted
set; all replications of all inputs go into one gm_sketch call per k.  The truth
is computed on the host from the definitions: J_P (Sec. 1) and c = sum v.  The
theory to compare with: Var(J^) = J_P (1 - J_P) / k (Sec. 2.4) and, for
c^ = (k - 1) / sum_j y_j with sum_j y_j ~ Gamma(k, c), Var(c^ / c) = 1 / (k - 2).
"""
import math

import numpy as np
import torch

from . import gm
from .workloads import CSR, ID_SPACE, from_rows, jaccard_pairs

REP_SHIFT = ID_SPACE  # ids of replication r are id + r 2^24 (r < 128 keeps them below 2^31)


def probability_jaccard(ia, wa, ib, wb):
    """J_P(u, v) = sum over ids positive in both of 1 / sum_l max(u_l / u_i, v_l / v_i)."""
    ids = np.union1d(ia, ib)
    u = np.zeros(ids.size)
    v = np.zeros(ids.size)
    u[np.searchsorted(ids, ia)] = wa
    v[np.searchsorted(ids, ib)] = wb
    both = np.nonzero((u > 0) & (v > 0))[0]
    total = 0.0
    for i in both:
        total += 1.0 / np.sum(np.maximum(u / u[i], v / v[i]))
    return total


def _replicate(X, reps):
    """reps copies of every row of X, copy r with ids shifted by r 2^24 (rows ordered rep-major)."""
    if reps > 127 or (X.nnz and int(X.ids.max()) >= REP_SHIFT):
        raise ValueError("replication needs ids < 2^24 and at most 127 copies")
    rows = []
    for r in range(reps):
        for i in range(X.n_rows):
            lo, hi = X.row_ptr[i], X.row_ptr[i + 1]
            rows.append(((X.ids[lo:hi].astype(np.int64) + r * REP_SHIFT).astype(np.int32), X.w[lo:hi]))
    return from_rows(rows)


def jaccard_rmse(ks=(64, 128, 256, 512, 1024, 2048, 4096), n_pairs=40, n_pos=1000, reps=32, shared=0.5,
                 seed=1, sketch_seed=7):
    """Task 1: RMSE of J^ over pairs and replications against the theory, per k."""
    A, B = jaccard_pairs(seed, n_pairs, n_pos, shared=shared)
    J = np.array([probability_jaccard(A.ids[A.row_ptr[p]:A.row_ptr[p + 1]], A.w[A.row_ptr[p]:A.row_ptr[p + 1]],
                                      B.ids[B.row_ptr[p]:B.row_ptr[p + 1]], B.w[B.row_ptr[p]:B.row_ptr[p + 1]])
                  for p in range(n_pairs)])
    Ar, Br = gm.to_device(_replicate(A, reps)), gm.to_device(_replicate(B, reps))
    out = []
    for k in ks:
        sa, _, _ = gm.gm_sketch(*Ar, k, sketch_seed)
        sb, _, _ = gm.gm_sketch(*Br, k, sketch_seed)
        est = gm.gm_jaccard(sa, sb).cpu().numpy().reshape(reps, n_pairs)
        err = est - J[None, :]
        out.append({"k": k, "rmse": float(np.sqrt(np.mean(err ** 2))),
                    "theory": float(np.sqrt(np.mean(J * (1 - J) / k))), "bias": float(np.mean(err))})
    return {"pairs": n_pairs, "n_pos": n_pos, "replications": reps, "mean_J": float(J.mean()), "by_k": out}


def weights(rng, n, kind):
    """UNI(0,1] or N(1, 0.1) (resampled until positive) weights."""
    if kind == "uniform":
        return 1.0 - rng.random(n)
    w = rng.normal(1.0, 0.1, n)
    while (w <= 0).any():
        bad = w <= 0
        w[bad] = rng.normal(1.0, 0.1, int(bad.sum()))
    return w


def cardinality_rmse(ks=(64, 256, 1024, 4096), ns=(100, 1000, 10000, 100000), kinds=("uniform", "normal"),
                     reps=64, seed=2, sketch_seed=9):
    """Task 2: relative RMSE of c^ = (k - 1) / sum y over replications against 1 / sqrt(k - 2)."""
    rng = np.random.default_rng(seed)
    out = []
    for kind in kinds:
        for n in ns:
            ids = rng.choice(ID_SPACE, n, replace=False).astype(np.int32)
            w = weights(rng, n, kind)
            c = math.fsum(w)
            X = _replicate(CSR(np.array([0, n], dtype=np.int64), ids, w), reps)
            dev = gm.to_device(X)
            for k in ks:
                _, y, _ = gm.gm_sketch(*dev, k, sketch_seed)
                est = gm.gm_cardinality(y).cpu().numpy()
                rel = est / c - 1.0
                out.append({"weights": kind, "n": n, "k": k, "rel_rmse": float(np.sqrt(np.mean(rel ** 2))),
                            "theory": 1.0 / math.sqrt(k - 2), "bias": float(np.mean(rel))})
    return {"replications": reps, "rows": out}
