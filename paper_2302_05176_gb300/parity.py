"""Comparison of a GPU sketch with a reference sketch, under the tolerance the
sketch's definition allows (pure numpy; no arithmetic of the sketch itself).

Register values may differ by at most `max_ulp` units in the last place: the
two sides compute the same exact sums and correctly rounded products, and differ
only in the natural logarithm (each within about one ulp).  Register indices
must be equal, except where the reference's two smallest candidate arrivals lie
within `tie_rel` of each other (a near-tie, which a one-ulp difference in a
logarithm can flip); those registers are counted and only checked to be within
`tie_rel`.
"""
import numpy as np


def ulp_distance(a, b):
    """|bits(a) - bits(b)| for non-negative doubles (inf == inf gives 0)."""
    ia = np.asarray(a, dtype=np.float64).view(np.int64)
    ib = np.asarray(b, dtype=np.float64).view(np.int64)
    return np.abs(ia - ib)


def compare_sketch(s, y, s_ref, y_ref, y2_ref=None, max_ulp=4, tie_rel=1e-12):
    s = np.asarray(s).reshape(np.shape(s_ref))
    y = np.asarray(y).reshape(np.shape(y_ref))
    filled_ref = np.isfinite(y_ref)
    filled = np.isfinite(y)
    rep = {"registers": int(np.size(y_ref))}
    if not np.array_equal(filled, filled_ref):
        rep.update(ok=False, reason="filled pattern differs", n_bad=int(np.sum(filled != filled_ref)))
        return rep
    if np.any(s[~filled] != -1) or np.any(s_ref[~filled_ref] != -1):
        rep.update(ok=False, reason="unfilled register with an id")
        return rep
    if y2_ref is None:
        tie = np.zeros_like(filled_ref)
    else:
        with np.errstate(invalid="ignore", divide="ignore"):
            tie = filled_ref & np.isfinite(y2_ref) & ((y2_ref - y_ref) <= tie_rel * y_ref)
    d = ulp_distance(y, y_ref)
    d[~filled_ref] = 0
    plain = filled_ref & ~tie
    bad_idx = plain & (s != s_ref)
    bad_val = plain & (d > max_ulp)
    with np.errstate(invalid="ignore"):
        bad_tie = tie & (np.abs(y - y_ref) > 2 * tie_rel * y_ref)
    rep.update(
        ok=not (bad_idx.any() or bad_val.any() or bad_tie.any()),
        max_ulp=int(d[plain].max()) if plain.any() else 0,
        mean_ulp=float(d[plain].mean()) if plain.any() else 0.0,
        near_ties=int(tie.sum()),
        tie_index_flips=int((tie & (s != s_ref)).sum()),
        index_mismatches=int(bad_idx.sum()),
        value_mismatches=int(bad_val.sum()),
    )
    if not rep["ok"]:
        where = np.argwhere(bad_idx | bad_val | bad_tie)[:5]
        rep["examples"] = [(tuple(int(v) for v in w), int(s[tuple(w)]), int(s_ref[tuple(w)]),
                            float(y[tuple(w)]), float(y_ref[tuple(w)])) for w in where]
    return rep
