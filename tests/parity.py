"""Comparison of a GPU sketch with the oracle's, under the tolerance the sketch's
definition allows (test infrastructure: pure numpy, no arithmetic of the sketch).

Register values may differ by at most `max_ulp` units in the last place: the two
sides compute the same exact sums and correctly rounded products, and differ
only in the natural logarithm (each within about half an ulp).

Register ids must be equal, with one exception: where the oracle's two best
candidates in the register (its winner and its runner-up, Eq. sjv) lie within
`tie_rel` of each other, an ulp in a logarithm can reverse their order.  Such a
register (a near-tie) may hold the runner-up instead, and then its value must be
within `max_ulp` of the runner-up's time.  Every register, near-tie or not, is
held to `max_ulp` against the candidate whose id it carries.
"""
import numpy as np


def ulp_distance(a, b):
    """|bits(a) - bits(b)| for non-negative doubles (inf == inf gives 0)."""
    ia = np.asarray(a, dtype=np.float64).view(np.int64)
    ib = np.asarray(b, dtype=np.float64).view(np.int64)
    return np.abs(ia - ib)


def compare_sketch(s, y, s_ref, y_ref, y2_ref=None, s2_ref=None, max_ulp=4, tie_rel=1e-12):
    """s, y: the sketch under test; s_ref, y_ref: the oracle's; y2_ref, s2_ref: the
    oracle's runner-up times and ids (oracle.sketch(..., runner_up=True)), or None
    to demand equal ids everywhere."""
    s_ref = np.asarray(s_ref)
    y_ref = np.asarray(y_ref)
    s = np.asarray(s).reshape(s_ref.shape)
    y = np.asarray(y).reshape(y_ref.shape)
    if (y2_ref is None) != (s2_ref is None):
        raise ValueError("the runner-up needs both its times and its ids")
    filled_ref = np.isfinite(y_ref)
    filled = np.isfinite(y)
    rep = {"registers": int(y_ref.size)}
    if not np.array_equal(filled, filled_ref):
        rep.update(ok=False, reason="filled pattern differs", n_bad=int(np.sum(filled != filled_ref)))
        return rep
    if np.any(s[~filled] != -1) or np.any(s_ref[~filled_ref] != -1):
        rep.update(ok=False, reason="unfilled register with an id")
        return rep
    if y2_ref is None:
        tie = np.zeros_like(filled_ref)
        y2_ref = np.full_like(y_ref, np.inf)
        s2_ref = np.full_like(s_ref, -1)
    else:
        y2_ref = np.asarray(y2_ref).reshape(y_ref.shape)
        s2_ref = np.asarray(s2_ref).reshape(s_ref.shape)
        with np.errstate(invalid="ignore", divide="ignore"):
            tie = filled_ref & np.isfinite(y2_ref) & ((y2_ref - y_ref) <= tie_rel * y_ref)
    same = filled_ref & (s == s_ref)
    flip = filled_ref & tie & (s != s_ref) & (s == s2_ref)  # the runner-up won the near-tie
    d = np.zeros(y_ref.shape, dtype=np.int64)
    d[same] = ulp_distance(y[same], y_ref[same])
    d[flip] = ulp_distance(y[flip], y2_ref[flip])
    bad_idx = filled_ref & ~same & ~flip
    bad_val = (same | flip) & (d > max_ulp)
    checked = same | flip
    rep.update(
        ok=not (bad_idx.any() or bad_val.any()),
        max_ulp=int(d[checked].max()) if checked.any() else 0,
        mean_ulp=float(d[checked].mean()) if checked.any() else 0.0,
        near_ties=int(tie.sum()),
        tie_index_flips=int(flip.sum()),
        index_mismatches=int(bad_idx.sum()),
        value_mismatches=int(bad_val.sum()),
    )
    if not rep["ok"]:
        where = np.argwhere(bad_idx | bad_val)[:5]
        rep["examples"] = [(tuple(int(v) for v in w), int(s[tuple(w)]), int(s_ref[tuple(w)]),
                            int(s2_ref[tuple(w)]), float(y[tuple(w)]), float(y_ref[tuple(w)]),
                            float(y2_ref[tuple(w)])) for w in where]
    return rep
