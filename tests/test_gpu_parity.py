"""CUDA path (through the C-ABI) against the CPU oracle, element by element.

Tolerance (from the definition in include/gm.h): both sides form the same exact
sums and correctly rounded products and differ only in ln(u); register ids agree
exactly and values within 4 ulp, except at near-ties (the oracle's winner and
runner-up within 1e-12 relative), where the register may hold the runner-up, its
value then within 4 ulp of the runner-up's time (tests/parity.py).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_05176_gb300 import gm
from paper_2302_05176_gb300 import workloads as W
from parity import compare_sketch

pytestmark = pytest.mark.gpu


def run(fn, X, k, seed, flags=gm.GM_FLAG_VALIDATE):
    rp, ids, w = gm.to_device(X)
    s, y, ws = fn(rp, ids, w, k, seed, flags=flags)
    code, stats = gm.gm_status(ws)
    assert code == gm.GM_OK, gm.strerror(code)
    return s.cpu().numpy(), y.cpu().numpy(), stats


def check(X, k, seed, flags=gm.GM_FLAG_VALIDATE, variants=("fastgm", "plain", "fastgm_fp64", "fastgm_int")):
    """Every variant against the oracle; FastGM and plain bit-identical within one arithmetic,
    and the default (mixed) and all-integer arithmetics bit-identical to each other."""
    s_ref, y_ref, y2_ref, s2_ref = oracle.sketch(X.row_ptr, X.ids, X.w, k, seed, runner_up=True)
    table = {"fastgm": (gm.gm_sketch, 0), "plain": (gm.gm_sketch_plain, 0),
             "fastgm_fp64": (gm.gm_sketch, gm.GM_FLAG_FP64_UNIT), "plain_fp64": (gm.gm_sketch_plain, gm.GM_FLAG_FP64_UNIT),
             "fastgm_int": (gm.gm_sketch, gm.GM_FLAG_INT_PRODUCTS),
             "plain_int": (gm.gm_sketch_plain, gm.GM_FLAG_INT_PRODUCTS)}
    outs = {}
    for name in variants:
        fn, extra = table[name]
        f = (flags if fn is gm.gm_sketch else flags & gm.GM_FLAG_VALIDATE) | extra
        s, y, stats = run(fn, X, k, seed, flags=f)
        rep = compare_sketch(s, y, s_ref, y_ref, y2_ref, s2_ref)
        assert rep["ok"], (name, rep)
        outs[name] = (s, y, stats, rep)
    for a, b in (("fastgm", "plain"), ("fastgm_fp64", "plain_fp64"), ("fastgm", "fastgm_int"), ("plain", "plain_int")):
        if a in outs and b in outs:
            assert np.array_equal(outs[a][0], outs[b][0])
            assert np.array_equal(outs[a][1].view(np.int64), outs[b][1].view(np.int64))
    return outs


def test_single_vector_k128():
    X = W.single_vector(seed=1)
    outs = check(X, 128, 1, variants=("fastgm", "plain", "fastgm_fp64", "plain_fp64", "fastgm_int", "plain_int"))
    assert outs["fastgm"][2]["arrivals"] < 0.2 * outs["plain"][2]["arrivals"]  # FastGM prunes


@pytest.mark.parametrize("k", [1, 2, 7, 31, 32, 33, 64, 257, 1024])
def test_ragged_rows(k):
    rng = np.random.default_rng(k)
    lens = [0, 1, 2, 3, 5, 17, 31, 32, 33, 100, 255, 256, 257, 600, 1500]
    rows = []
    for i, n in enumerate(lens):
        ids = np.sort(rng.choice(1 << 24, size=n, replace=False)).astype(np.int32)
        if i % 3 == 0:
            wts = 1.0 - rng.random(n)
        elif i % 3 == 1:
            wts = rng.standard_exponential(n)
        else:
            wts = W.pareto_weights(rng, n, 1.2, 1e-3)
        rows.append((ids, wts))
    check(W.from_rows(rows), k, 1234 + k)


@pytest.mark.parametrize("k", [256, 4096])
def test_lognormal_small_batch(k):
    X = W.lognormal_batch(seed=5, n_rows=24, median=300.0, hi=3000)
    check(X, k, 77)


def test_edge_weights_and_ids():
    rows = [
        (np.array([0], np.int32), np.array([1.0])),                                  # single element, id 0
        (np.array([5, 6, 7], np.int32), np.array([0.0, 0.0, 0.0])),                  # all zero -> unfilled
        (np.array([2**31 - 1, 3], np.int32), np.array([1e-300, 1e300])),             # extreme weights
        (np.array([10, 11, 12, 13], np.int32), np.array([1.0, 1e-12, 1e12, 0.5])),  # dynamic range
        (np.array([], np.int32), np.array([])),                                      # empty row
        (np.array([9, 8], np.int32), np.array([2.0, 2.0])),                          # unsorted ids
    ]
    for k in (1, 3, 64, 1000):
        check(W.from_rows(rows), k, 99)


def test_tight_bound_escalations_agree():
    """Shrunken first-pass bounds force escalations: same registers, more passes."""
    X = W.lognormal_batch(seed=13, n_rows=32, median=300.0, hi=4000)
    outs = check(X, 512, 21, flags=gm.GM_FLAG_VALIDATE | gm.GM_FLAG_TIGHT_BOUND, variants=("fastgm",))
    assert outs["fastgm"][2]["rows_escalated"] > 0


@pytest.mark.parametrize("tight", [0, gm.GM_FLAG_TIGHT_BOUND])
def test_long_rows_split_into_chunks(tight):
    """Rows longer than 32,768 elements are cut into chunks sketched by different CTAs
    and merged (Sec. 2.3 union); with a tight bound they are also redone whole."""
    rng = np.random.default_rng(17)
    rows = []
    for n in (70_000, 33_000, 5, 40_000, 1200):
        ids = np.sort(rng.choice(1 << 24, size=n, replace=False)).astype(np.int32)
        rows.append((ids, W.pareto_weights(rng, n, 1.2, 1e-3)))
    X = W.from_rows(rows)
    outs = check(X, 128, 5, flags=gm.GM_FLAG_VALIDATE | tight, variants=("fastgm", "plain"))
    if tight:
        assert outs["fastgm"][2]["rows_escalated"] >= 0


@pytest.mark.parametrize("tight", [0, gm.GM_FLAG_TIGHT_BOUND])
def test_wide_shape_long_rows_and_escalations(tight):
    """k = 4096 runs 1024-thread CTAs: long rows cut into chunks merged across CTAs
    and, with a shrunken bound, rows redone by the escalation kernel.  The registers
    equal the plain sketch's and the 512-thread shape's (the all-integer arithmetic
    runs there), bit for bit."""
    rng = np.random.default_rng(23)
    rows = []
    for n in [70_000, 33_000, 5, 40_000, 1200] + [int(x) for x in rng.integers(1, 3000, 40)]:
        ids = np.sort(rng.choice(1 << 24, size=n, replace=False)).astype(np.int32)
        rows.append((ids, W.pareto_weights(rng, n, 1.2, 1e-3) if n > 2000 else rng.standard_exponential(n)))
    X = W.from_rows(rows)
    k = 4096
    f = gm.GM_FLAG_VALIDATE | tight
    s0, y0, st0 = run(gm.gm_sketch, X, k, 31, flags=f)
    s1, y1, _ = run(gm.gm_sketch, X, k, 31, flags=f | gm.GM_FLAG_INT_PRODUCTS)
    s2, y2, _ = run(gm.gm_sketch_plain, X, k, 31)
    for s, y in ((s1, y1), (s2, y2)):
        assert np.array_equal(s0, s) and np.array_equal(y0.view(np.int64), y.view(np.int64))
    if tight:
        assert st0["rows_escalated"] > 0


@pytest.mark.parametrize("tight", [0, gm.GM_FLAG_TIGHT_BOUND])
def test_compacted_long_rows_against_oracle(tight):
    """Long rows compacted (GM_FLAG_COMPACT_LONG: this batch is below the size at
    which they are by default): screened first by the whole grid, then sketched
    from the compact lists of the elements left; with a tight bound also redone
    whole.  Against the oracle at k = 128."""
    rng = np.random.default_rng(29)
    rows = []
    for n in (70_000, 33_000, 40_000):
        ids = np.sort(rng.choice(1 << 24, size=n, replace=False)).astype(np.int32)
        rows.append((ids, W.pareto_weights(rng, n, 1.2, 1e-3)))
    X = W.from_rows(rows)
    outs = check(X, 128, 9, flags=gm.GM_FLAG_VALIDATE | gm.GM_FLAG_COMPACT_LONG | tight,
                 variants=("fastgm", "plain"))
    assert outs["fastgm"][2]["arrivals"] < 0.1 * outs["plain"][2]["arrivals"]


@pytest.mark.parametrize("k", [1024, 4096])
def test_long_rows_heavy_and_super_heavy_elements(k):
    """Long rows compacted (screened first by the whole grid, then sketched from
    their compact lists; GM_FLAG_COMPACT_LONG) with planted elements whose expected arrivals below the bound exceed
    the heavy threshold (warp-path units, with the medium ones) and the super-heavy one
    (an element streamed by a whole CTA, up to all k arrivals), against the oracle
    and bit for bit against the plain sketch."""
    rng = np.random.default_rng(59 + k)
    rows = []
    for n in ((40_000, 34_000) if k == 1024 else (36_000,)):
        ids = np.sort(rng.choice(1 << 24, size=n, replace=False)).astype(np.int32)
        w = rng.standard_exponential(n)
        total = w.sum()
        pos = rng.choice(n, size=12, replace=False)
        w[pos[:4]] = total * np.array([0.3, 0.1, 0.05, 0.02])  # super-heavy: hundreds to all k arrivals
        w[pos[4:]] = total * rng.uniform(0.004, 0.01, size=8)   # heavy: about 60 to 250 arrivals
        rows.append((ids, w))
    X = W.from_rows(rows)
    s0, y0, st0 = run(gm.gm_sketch, X, k, 7, flags=gm.GM_FLAG_VALIDATE | gm.GM_FLAG_COMPACT_LONG)
    s1, y1, _ = run(gm.gm_sketch_plain, X, k, 7)
    s2, y2, _ = run(gm.gm_sketch, X, k, 7)  # the element ranges (the batch is small)
    assert np.array_equal(s0, s2) and np.array_equal(y0.view(np.int64), y2.view(np.int64))
    assert np.array_equal(s0, s1) and np.array_equal(y0.view(np.int64), y1.view(np.int64))
    s_ref, y_ref, y2_ref, s2_ref = oracle.sketch_rows_parallel(X.row_ptr, X.ids, X.w, k, 7,
                                                               np.arange(X.n_rows), runner_up=True)
    rep = compare_sketch(s0, y0, s_ref, y_ref, y2_ref, s2_ref)
    assert rep["ok"], rep
    assert st0["heavy_elements"] >= 12


def test_bound_modes_agree():
    """FastGM without an initial bound (FastSearch's doubling horizon from 1/sum v,
    long-row chunks pruned by the row's merged y*) gives the closed form's
    registers; it keeps more arrivals, but of the same order (not the k n+ of the
    unpruned stream)."""
    X = W.lognormal_batch(seed=9, n_rows=16, median=400.0, hi=2000)
    k = 512
    s0, y0, st0 = run(gm.gm_sketch, X, k, 3, flags=gm.GM_BOUND_CLOSED)
    s1, y1, st1 = run(gm.gm_sketch, X, k, 3, flags=gm.GM_BOUND_NONE)
    assert np.array_equal(s0, s1) and np.array_equal(y0.view(np.int64), y1.view(np.int64))
    assert st0["kept"] < st1["kept"] < 4 * st0["kept"]
    assert st1["kept"] < 0.2 * k * X.nnz


@pytest.mark.parametrize("k", [128, 4096])
def test_bound_free_long_rows_against_oracle(k):
    """The bound-free mode on rows cut into chunks (each chunk grows its own bound
    until its registers fill or the row's merged y* is finite) and on short rows,
    against the oracle; at k = 4096 against the plain sketch too."""
    rng = np.random.default_rng(41)
    rows = []
    for n in (70_000, 33_000, 5, 40_000, 1200, 0, 1):
        ids = np.sort(rng.choice(1 << 24, size=n, replace=False)).astype(np.int32)
        rows.append((ids, W.pareto_weights(rng, n, 1.2, 1e-3) if n % 2 else rng.standard_exponential(n)))
    X = W.from_rows(rows)
    if k == 128:
        check(X, k, 5, flags=gm.GM_FLAG_VALIDATE | gm.GM_BOUND_NONE, variants=("fastgm", "fastgm_int"))
    else:
        s0, y0, st0 = run(gm.gm_sketch, X, k, 5, flags=gm.GM_FLAG_VALIDATE | gm.GM_BOUND_NONE)
        s1, y1, _ = run(gm.gm_sketch_plain, X, k, 5)
        assert np.array_equal(s0, s1) and np.array_equal(y0.view(np.int64), y1.view(np.int64))
        sub = np.array([2, 4, 6])  # the short rows against the oracle
        s_ref, y_ref, y2_ref, s2_ref = oracle.sketch_rows_parallel(X.row_ptr, X.ids, X.w, k, 5, sub,
                                                                   runner_up=True)
        rep = compare_sketch(s0[sub], y0[sub], s_ref, y_ref, y2_ref, s2_ref)
        assert rep["ok"], rep


def test_seed_changes_sketch_and_repeat_is_deterministic():
    X = W.lognormal_batch(seed=2, n_rows=8, median=200.0, hi=800)
    a = run(gm.gm_sketch, X, 256, 1)
    b = run(gm.gm_sketch, X, 256, 1)
    c = run(gm.gm_sketch, X, 256, 2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1].view(np.int64), b[1].view(np.int64))
    assert not np.array_equal(a[0], c[0])


def test_validation_reports_bad_data():
    ws = gm.workspace(1, 1000, 16)  # big enough for every call below
    for ids_, w_ in (([1, 2], [1.0, -2.0]), ([1, -2], [1.0, 2.0]), ([1, 2], [1.0, float("nan")]),
                     ([1, 2], [float("inf"), 1.0])):
        bad = W.from_rows([(np.array(ids_, np.int32), np.array(w_))])
        rp, ids, w = gm.to_device(bad)
        gm.gm_sketch(rp, ids, w, 16, 1, flags=gm.GM_FLAG_VALIDATE, ws=ws)
        assert gm.gm_status(ws)[0] == gm.GM_EDATA
    # row_ptr that does not end at nnz
    rp = torch.tensor([0, 1], dtype=torch.int64, device="cuda")
    ids = torch.tensor([3, 4], dtype=torch.int32, device="cuda")
    w = torch.tensor([1.0, 1.0], dtype=torch.float64, device="cuda")
    gm.gm_sketch(rp, ids, w, 16, 1, flags=gm.GM_FLAG_VALIDATE, ws=ws)
    assert gm.gm_status(ws)[0] == gm.GM_EDATA
    # a good call through the same workspace is clean again
    good = W.single_vector(seed=3)
    rp, ids, w = gm.to_device(good)
    gm.gm_sketch(rp, ids, w, 16, 1, flags=gm.GM_FLAG_VALIDATE, ws=ws)
    assert gm.gm_status(ws)[0] == gm.GM_OK


def test_host_errors():
    X = W.single_vector(seed=1)
    rp, ids, w = gm.to_device(X)
    with pytest.raises(gm.GmError):
        gm.gm_sketch(rp, ids, w, 0, 1)
    with pytest.raises(gm.GmError):
        gm.gm_sketch(rp, ids, w, gm.GM_MAX_K + 1, 1)
    tiny = torch.empty(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(gm.GmError):
        gm.gm_sketch(rp, ids, w, 16, 1, ws=tiny)
    # a workspace off the 256-byte boundary is refused before any launch
    big = torch.empty(gm.lib().gm_sketch_workspace_bytes(1, X.nnz, 16, 0) + 256, dtype=torch.uint8, device="cuda")
    for off in (16, 128):
        with pytest.raises(gm.GmError) as e:
            gm.gm_sketch(rp, ids, w, 16, 1, ws=big[off:])
        assert e.value.code == gm.GM_EINVAL
    gm.gm_sketch(rp, ids, w, 16, 1, ws=big[256:])


def test_estimators_against_oracle():
    A, B = W.jaccard_pairs(seed=4, n_pairs=40, n_pos=300)
    k = 256
    sa, ya, _ = run(gm.gm_sketch, A, k, 11)
    sb, yb, _ = run(gm.gm_sketch, B, k, 11)
    dev = "cuda"
    j = gm.gm_jaccard(torch.from_numpy(sa).to(dev), torch.from_numpy(sb).to(dev)).cpu().numpy()
    assert np.array_equal(j, oracle.jaccard(sa, sb))
    c = gm.gm_cardinality(torch.from_numpy(ya).to(dev)).cpu().numpy()
    c_ref = oracle.cardinality(ya)
    assert np.allclose(c, c_ref, rtol=k * 2.0 ** -52, atol=0)
    sm, ym = gm.gm_merge(torch.from_numpy(sa).to(dev), torch.from_numpy(ya).to(dev),
                         torch.from_numpy(sb).to(dev), torch.from_numpy(yb).to(dev))
    so, yo = oracle.merge(sa, ya, sb, yb)
    assert np.array_equal(sm.cpu().numpy(), so) and np.array_equal(ym.cpu().numpy(), yo)
    # an unfilled register estimates cardinality 0 and never collides
    y_unf = np.full((1, 8), np.inf)
    s_unf = np.full((1, 8), -1, np.int32)
    assert gm.gm_cardinality(torch.from_numpy(y_unf).to(dev)).item() == 0.0
    assert gm.gm_jaccard(torch.from_numpy(s_unf).to(dev), torch.from_numpy(s_unf).to(dev)).item() == 0.0


def test_merge_equals_union_on_gpu():
    rng = np.random.default_rng(3)
    ids = np.sort(rng.choice(1 << 20, size=3000, replace=False)).astype(np.int32)
    wts = rng.standard_exponential(3000)
    part = rng.random(3000) < 0.4
    A = W.from_rows([(ids[part], wts[part])])
    B = W.from_rows([(ids[~part], wts[~part])])
    U = W.from_rows([(ids, wts)])
    k = 1024
    sa, ya, _ = run(gm.gm_sketch, A, k, 5)
    sb, yb, _ = run(gm.gm_sketch, B, k, 5)
    su, yu, _ = run(gm.gm_sketch, U, k, 5)
    dev = "cuda"
    sm, ym = gm.gm_merge(*(torch.from_numpy(x).to(dev) for x in (sa, ya, sb, yb)))
    assert np.array_equal(sm.cpu().numpy(), su) and np.array_equal(ym.cpu().numpy(), yu)


def test_lognormal_batch_full_size_sampled_rows():
    """4,096 rows, n+ ~ LogNormal(ln 2000, 1) clipped to [10, 2e5], Exp(1), k = 1024, seed 1:
    the launch the benchmark times; sampled rows against the oracle, all rows by properties."""
    X = W.lognormal_batch(seed=1)
    k, seed = 1024, 1
    s, y, stats = run(gm.gm_sketch, X, k, seed, flags=0)
    lens = np.diff(X.row_ptr)
    order = np.argsort(lens)
    rng = np.random.default_rng(0)
    sample = np.unique(np.concatenate([order[:4], rng.choice(np.flatnonzero(lens < 4000), size=6, replace=False)]))
    s_ref, y_ref, y2_ref, s2_ref = oracle.sketch_rows_parallel(X.row_ptr, X.ids, X.w, k, seed, sample,
                                                               runner_up=True)
    rep = compare_sketch(s[sample], y[sample], s_ref, y_ref, y2_ref, s2_ref)
    assert rep["ok"], rep
    # properties on every row: all registers filled, ids drawn from the row, times positive
    assert np.all(np.isfinite(y)) and np.all(y > 0)
    for r in rng.choice(X.n_rows, size=64, replace=False):
        assert np.isin(s[r], X.row(r)[0]).all()


def test_lognormal_batch_full_size_k4096_sampled_rows():
    """The same 4,096-row batch at k = 4096, the benchmark's second launch (1024-thread
    CTAs): sampled rows against the oracle, every row bit-identical to the
    512-thread shape (the all-integer arithmetic runs there), all registers filled."""
    X = W.lognormal_batch(seed=1)
    k, seed = 4096, 1
    s, y, _ = run(gm.gm_sketch, X, k, seed, flags=0)
    s_i, y_i, _ = run(gm.gm_sketch, X, k, seed, flags=gm.GM_FLAG_INT_PRODUCTS)
    assert np.array_equal(s, s_i) and np.array_equal(y.view(np.int64), y_i.view(np.int64))
    lens = np.diff(X.row_ptr)
    order = np.argsort(lens)
    rng = np.random.default_rng(1)
    sample = np.unique(np.concatenate([order[:3], rng.choice(np.flatnonzero(lens < 1500), size=4, replace=False)]))
    s_ref, y_ref, y2_ref, s2_ref = oracle.sketch_rows_parallel(X.row_ptr, X.ids, X.w, k, seed, sample,
                                                               runner_up=True)
    rep = compare_sketch(s[sample], y[sample], s_ref, y_ref, y2_ref, s2_ref)
    assert rep["ok"], rep
    assert np.all(np.isfinite(y)) and np.all(y > 0)


def _batch_rows_against_oracle(k, rows, seed=1):
    """The 4,096-row benchmark batch sketched as the benchmark launches it (flags 0,
    k registers), the listed rows against the unpruned oracle with its runner-ups."""
    X = W.lognormal_batch(seed=seed)
    s, y, _ = run(gm.gm_sketch, X, k, seed, flags=0)
    s_ref, y_ref, y2_ref, s2_ref = oracle.sketch_rows_parallel(X.row_ptr, X.ids, X.w, k, seed, rows,
                                                               runner_up=True)
    rep = compare_sketch(s[rows], y[rows], s_ref, y_ref, y2_ref, s2_ref)
    assert rep["ok"], rep
    return rep


def test_lognormal_batch_long_rows_k1024():
    """Every row of the benchmark batch longer than 32,768 elements (13 rows, 34,538 to
    85,181 elements: cut into chunks, merged by the global (y, id) minimum, redone
    whole when a chunk pass leaves a register unfilled), and eight rows of 4,000 to
    32,768 elements, against the oracle at the benchmark's k = 1024."""
    X = W.lognormal_batch(seed=1)
    lens = np.diff(X.row_ptr)
    long_rows = np.flatnonzero(lens > 32768)
    assert long_rows.size == 13
    rng = np.random.default_rng(2)
    mid = rng.choice(np.flatnonzero((lens >= 4000) & (lens <= 32768)), size=8, replace=False)
    _batch_rows_against_oracle(1024, np.sort(np.concatenate([long_rows, mid])))


def test_lognormal_batch_long_rows_k4096():
    """The benchmark batch at k = 4096 (1024-thread CTAs): its two shortest rows over
    32,768 elements (chunked) and ten rows of 4,000 to 32,768 elements against the
    oracle."""
    X = W.lognormal_batch(seed=1)
    lens = np.diff(X.row_ptr)
    long_rows = np.flatnonzero(lens > 32768)
    two = long_rows[np.argsort(lens[long_rows])[:2]]
    rng = np.random.default_rng(3)
    mid = rng.choice(np.flatnonzero((lens >= 4000) & (lens <= 32768)), size=10, replace=False)
    _batch_rows_against_oracle(4096, np.sort(np.concatenate([two, mid])))


def test_pareto_heavy_full_size():
    """16 rows x 10^6 elements, Pareto(1.2, x_min 1e-3), k = 4096, seed 1: the heavy-tail
    launch the benchmark times.  FastGM equals the plain O(k n+) sketch on every
    register of every row, and row 0 equals the oracle's Algorithm 1."""
    X = W.pareto_heavy(seed=1)
    k, seed = 4096, 1
    rp, ids, w = gm.to_device(X)
    s, y, _ = gm.gm_sketch(rp, ids, w, k, seed)
    sp, yp, _ = gm.gm_sketch_plain(rp, ids, w, k, seed)
    assert torch.equal(s, sp) and torch.equal(y.view(torch.int64), yp.view(torch.int64))
    sn, yn, wsn = gm.gm_sketch(rp, ids, w, k, seed, flags=gm.GM_BOUND_NONE)
    assert torch.equal(s, sn) and torch.equal(y.view(torch.int64), yn.view(torch.int64))
    assert gm.gm_status(wsn)[1]["arrivals"] < 0.05 * X.nnz * k  # pruned, though without an initial bound
    lo, hi = X.row_ptr[0], X.row_ptr[1]
    s_ref, y_ref, _ = oracle.fastgm_alg1(X.ids[lo:hi], X.w[lo:hi], k, seed)
    rep = compare_sketch(s[0].cpu().numpy(), y[0].cpu().numpy(), s_ref, y_ref)
    assert rep["ok"], rep
