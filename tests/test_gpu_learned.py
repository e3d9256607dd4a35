"""The learned first-pass bound on the GPU against the FP64 oracle (oracle/mlp.py).

* row features, ln y*, network forward, pinball gradient and Adam step against
  the oracle on the same inputs; the gradient is the same bits on every call;
* gm_sketch_learned gives the registers of gm_sketch for ANY model (untrained,
  all-fallback, unbounded, NaN parameters), long rows included;
* a network trained by the library's own kernels: its fallback rate is near
  1 - tau, it lands on the closed-form quantile (the information limit), and it
  does far less work than FastGM without an initial bound.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import mlp
from paper_2302_05176_gb300 import gm, learned
from paper_2302_05176_gb300 import workloads as W
from parity import compare_sketch

pytestmark = pytest.mark.gpu


def edge_batch():
    rng = np.random.default_rng(21)
    rows = [
        (np.array([], dtype=np.int32), np.array([])),                                    # empty
        (np.array([3, 9], dtype=np.int32), np.array([0.0, -1.0])),                       # no positive weight
        (np.array([1, 2, 5], dtype=np.int32), np.array([5e-324, 1e300, 1.0])),          # extremes
        (np.arange(100, dtype=np.int32), np.ones(100)),                                  # equal weights
        (np.arange(7, dtype=np.int32), np.array([1.0, 2, 4, 8, 0, np.nan, np.inf])),     # skipped entries
        (rng.choice(1 << 24, 5000, replace=False).astype(np.int32), W.pareto_weights(rng, 5000, 1.2, 1e-3)),
    ]
    return W.from_rows(rows)


@pytest.mark.parametrize("k", [1, 256, 4096])
def test_features_match_oracle(k):
    X = W.lognormal_batch(seed=3, n_rows=48, median=300.0)
    sizes = W.uniform_rows(seed=4, n_rows=5, n_pos=np.array([4095, 4096, 4097, 20000, 70000]), weight="exp")
    for batch in (X, edge_batch(), sizes):  # warp rows, block rows (> 4096 elements), edge cases
        rp, ids, w = gm.to_device(batch)
        got = gm.gm_features(rp, ids, w, k).cpu().numpy()
        ref = mlp.features_rows(batch.row_ptr, batch.w, k).astype(np.float32)
        assert np.array_equal(got[:, 3:8], ref[:, 3:8])          # quantile bins and ln k: exact
        # ln n+ and ln max v exactly as rounded; ln sum v from an FP32 sum (relative error ~2^-24)
        assert np.allclose(got[:, [0, 2]], ref[:, [0, 2]], rtol=3e-7, atol=0)
        assert np.allclose(got[:, 1], ref[:, 1], rtol=3e-7, atol=2e-7)


def test_row_ln_ystar():
    X = edge_batch()
    rp, ids, w = gm.to_device(X)
    _, y, _ = gm.gm_sketch(rp, ids, w, 64, 5)
    got = gm.gm_row_ln_ystar(y).cpu().numpy()
    yn = y.cpu().numpy()
    with np.errstate(divide="ignore"):
        want = np.log(yn.max(axis=1)).astype(np.float32)
    assert np.array_equal(np.isinf(got), np.isinf(want)) and np.isinf(got[0]) and np.isinf(got[1])
    fin = np.isfinite(want)
    assert np.allclose(got[fin], want[fin], rtol=1e-6, atol=1e-7)


def random_params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, size=mlp.P)


def feats_like(rng, n):
    X = np.column_stack([rng.uniform(2, 12, n), rng.uniform(2, 12, n), rng.uniform(0, 3, n),
                         rng.uniform(-3, 0, n), rng.uniform(-1, 1, n), rng.uniform(0, 2, n),
                         rng.uniform(1, 3, n), np.log(rng.choice([256, 1024, 4096], n))])
    return X.astype(np.float32)


def to_dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def test_forward_matches_oracle():
    theta = random_params(1).astype(np.float32)
    X = feats_like(np.random.default_rng(2), 3001)
    got = gm.gm_model_forward(to_dev(theta), to_dev(X)).cpu().numpy()
    ref, _ = mlp.forward(theta.astype(np.float64), X.astype(np.float64))
    assert np.allclose(got, ref, rtol=1e-5, atol=2e-5), np.abs(got - ref).max()


@pytest.mark.parametrize("n", [1, 1000, 70001])
def test_grad_matches_oracle_and_is_deterministic(n):
    rng = np.random.default_rng(3)
    theta = random_params(4).astype(np.float32)
    X = feats_like(rng, n)
    pred, _ = mlp.forward(theta.astype(np.float64), X.astype(np.float64))
    t = (pred + rng.choice([-1, 1], n) * rng.uniform(0.05, 1.0, n)).astype(np.float32)  # away from the kink
    tau = 0.9
    g1, l1, ws = gm.gm_model_grad(to_dev(theta), to_dev(X), to_dev(t), tau)
    g2, l2, _ = gm.gm_model_grad(to_dev(theta), to_dev(X), to_dev(t), tau, ws=ws)
    g1, g2 = g1.cpu().numpy(), g2.cpu().numpy()
    assert np.array_equal(g1.view(np.int32), g2.view(np.int32)) and float(l1) == float(l2)
    loss, gref = mlp.loss_and_grad(theta.astype(np.float64), X.astype(np.float64), t.astype(np.float64), tau)
    assert abs(float(l1) - loss) <= 1e-5 * abs(loss) + 1e-7
    scale = np.abs(gref).max()
    assert np.allclose(g1, gref, rtol=1e-3, atol=2e-5 * scale), np.abs(g1 - gref).max() / scale


def test_adam_matches_oracle():
    rng = np.random.default_rng(5)
    theta = rng.normal(size=mlp.P).astype(np.float32)
    p = to_dev(theta)
    mom = torch.zeros(2 * mlp.P, dtype=torch.float32, device="cuda")
    th, m, v = theta.astype(np.float64), np.zeros(mlp.P), np.zeros(mlp.P)
    for step in range(1, 6):
        g = rng.normal(size=mlp.P).astype(np.float32)
        gm.gm_model_adam(p, mom, to_dev(g), 1e-2, step)
        th, m, v = mlp.adam_step(th, m, v, g.astype(np.float64), 1e-2, step)
    assert np.allclose(p.cpu().numpy(), th, rtol=1e-5, atol=1e-6)


def test_init_save_load(tmp_path):
    a = gm.gm_model_init(42).cpu().numpy()
    b = gm.gm_model_init(42).cpu().numpy()
    c = gm.gm_model_init(43).cpu().numpy()
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    W1, b1, W2, b2, w3, b3 = mlp.unpack(a)
    assert np.all(np.abs(W1) <= 1 / math.sqrt(8)) and np.all(np.abs(W2) <= 0.125) and np.all(np.abs(w3) <= 0.125)
    assert not b1.any() and not b2.any() and b3 == 0
    assert abs(W1.mean()) < 0.05 and W1.std() > 0.15
    path = str(tmp_path / "bound.gmmlp")
    gm.gm_model_save(torch.from_numpy(a).cuda(), path)
    assert np.array_equal(gm.gm_model_load(path).cpu().numpy(), a)
    with pytest.raises(gm.GmError) as e:
        gm.gm_model_load(str(tmp_path / "missing"))
    assert e.value.code == gm.GM_EINVAL
    bad = tmp_path / "bad"
    bad.write_bytes(b"NOTAMODEL" + bytes(100))
    with pytest.raises(gm.GmError) as e:
        gm.gm_model_load(str(bad))
    assert e.value.code == gm.GM_EDATA


def long_batch():
    rng = np.random.default_rng(8)
    lens = [40000, 5, 3000, 0, 70000, 1, 200]
    rows = []
    for n in lens:
        w = rng.exponential(size=n)
        if n == 70000:
            w = W.pareto_weights(rng, n, 1.2, 1e-3)
        rows.append((rng.choice(1 << 24, n, replace=False).astype(np.int32), w))
    return W.from_rows(rows)


@pytest.mark.parametrize("k", [64, 1024, 4096])
def test_learned_sketch_exact_for_any_model(k):
    X = long_batch()
    rp, ids, w = gm.to_device(X)
    s0, y0, _ = gm.gm_sketch(rp, ids, w, k, 77)
    rand = gm.gm_model_init(9)
    nanp = rand.clone()
    nanp[100] = float("nan")
    zero = torch.zeros_like(rand)
    for params, margin in ((rand, 0.0), (rand, -30.0), (rand, 30.0), (nanp, 0.0), (zero, 0.0), (zero, -80.0)):
        s, y, ws = gm.gm_sketch_learned(rp, ids, w, k, 77, params, margin, flags=gm.GM_FLAG_VALIDATE)
        code, st = gm.gm_status(ws)
        assert code == gm.GM_OK
        assert torch.equal(s, s0) and torch.equal(y.view(torch.int64), y0.view(torch.int64)), (margin,)
        if margin == -30.0:
            assert st["rows_fallback"] == 6  # every row with a positive weight falls back (2 long)
        # the long rows compacted at the learned bound (screened by it first): the same registers
        s, y, ws = gm.gm_sketch_learned(rp, ids, w, k, 77, params, margin,
                                        flags=gm.GM_FLAG_VALIDATE | gm.GM_FLAG_COMPACT_LONG)
        assert gm.gm_status(ws)[0] == gm.GM_OK
        assert torch.equal(s, s0) and torch.equal(y.view(torch.int64), y0.view(torch.int64)), ("compact", margin)
    # and against the oracle on the short rows
    s_ref, y_ref, y2_ref, s2_ref = oracle.sketch_rows_parallel(X.row_ptr, X.ids, X.w, k, 77,
                                                               np.array([1, 2, 5, 6]), runner_up=True)
    rep = compare_sketch(s0.cpu().numpy()[[1, 2, 5, 6]], y0.cpu().numpy()[[1, 2, 5, 6]], s_ref, y_ref, y2_ref,
                         s2_ref)
    assert rep["ok"], rep


@pytest.mark.parametrize("k", [256, 4096])
def test_learned_bound_against_features_and_oracle(k):
    """gm_learned_bound: the same bits on every call; exp(gm_model_forward(gm_features)
    + margin) to the FP32 rounding of the exponential for rows of up to 2,048
    elements (the same feature code) and to that of a long row's sum beyond (its
    pieces are added in piece order); and the FP64 oracle's features and network."""
    rng = np.random.default_rng(41)
    lens = [0, 1, 2047, 2048, 2049, 4096, 8191, 8192, 8193, 16385, 30000, 120000]
    lens += [int(n) for n in rng.integers(1, 20000, 40)]
    rows = [(rng.choice(1 << 24, n, replace=False).astype(np.int32), rng.lognormal(0.0, 1.5, n)) for n in lens]
    rows[1] = (rows[1][0], np.array([0.0]))  # no positive weight
    X = W.from_rows(rows)
    rp, ids, w = gm.to_device(X)
    theta = random_params(6).astype(np.float32)
    params = to_dev(theta)
    margin = 0.25
    t1 = gm.gm_learned_bound(rp, w, k, params, margin)
    t2 = gm.gm_learned_bound(rp, w, k, params, margin)
    assert torch.equal(t1.view(torch.int32), t2.view(torch.int32))
    f = gm.gm_features(rp, ids, w, k)
    want = torch.exp(gm.gm_model_forward(params, f) + margin).cpu().numpy()
    got = t1.cpu().numpy()
    short = np.array([n <= 2048 for n in lens])
    assert np.allclose(got[short], want[short], rtol=3e-7, atol=0), np.abs(got / want - 1)[short].max()
    assert np.allclose(got[~short], want[~short], rtol=2e-5, atol=0), np.abs(got / want - 1)[~short].max()
    pred, _ = mlp.forward(theta.astype(np.float64), mlp.features_rows(X.row_ptr, X.w, k))
    assert np.allclose(got, np.exp(pred + margin), rtol=3e-4), np.abs(got / np.exp(pred + margin) - 1).max()


def test_learned_bound_overlapping_rows_stay_in_bounds():
    """Row offsets that do not ascend make rows overlap, so the long rows' pieces
    can outnumber the lists sized from nnz: such a row gets t = -1 (no learned
    bound, the closed form) and every other row its usual bound."""
    rng = np.random.default_rng(12)
    n = 100_000
    ids = torch.from_numpy(rng.choice(1 << 24, n, replace=False).astype(np.int32)).cuda()
    w = torch.from_numpy(rng.exponential(size=n)).cuda()
    params = gm.gm_model_init(5)
    full = torch.tensor([0, n], dtype=torch.int64, device="cuda")
    t_full = float(gm.gm_learned_bound(full, w, 256, params, 0.0)[0])
    rp = torch.tensor([0, n] * 10 + [0], dtype=torch.int64, device="cuda")  # rows 0, 2, ... span everything
    t = gm.gm_learned_bound(rp, w, 256, params, 0.0).cpu().numpy()
    full_rows, empty_rows = t[0::2], t[1::2]
    assert np.all((full_rows == -1.0) | (full_rows == t_full)), full_rows
    assert (full_rows == -1.0).any() and (full_rows == t_full).any()
    empty = torch.tensor([0, 0], dtype=torch.int64, device="cuda")
    t_empty = float(gm.gm_learned_bound(empty, w[:0], 256, params, 0.0)[0])
    assert np.all(empty_rows == t_empty)


def test_learned_bound_of_every_row_length():
    """Rows at the warp and piece limits (2,048 elements, and multiples of it) and long rows
    (their features gathered piece by piece over the grid) get the bound
    exp(gm_model_forward(gm_features) + margin): the number of
    rows whose learned pass falls back is the number predicted from gm_features,
    the network and the sketch's own y*, at several margins."""
    rng = np.random.default_rng(31)
    lens = [2047, 2048, 2049, 4095, 4096, 4097, 16384, 16385, 24577, 100000, 250000]
    lens += [int(n) for n in rng.integers(1, 60000, 29)]
    rows = [(rng.choice(1 << 24, n, replace=False).astype(np.int32), rng.lognormal(0.0, 2.0, n)) for n in lens]
    X = W.from_rows(rows)
    rp, ids, w = gm.to_device(X)
    k = 256
    s0, y0, _ = gm.gm_sketch(rp, ids, w, k, 5)
    params = gm.gm_model_init(3)
    f = gm.gm_features(rp, ids, w, k)
    pred = gm.gm_model_forward(params, f)  # the predicted ln bound (the network's output - ln sum v)
    ystar = y0.max(dim=1).values
    gaps = np.sort((torch.log(ystar) - pred.double()).cpu().numpy())
    for q in (3, 20, 36):
        margin = float(0.5 * (gaps[q] + gaps[q + 1]))  # between two rows: no decision sits on the edge
        s, y, ws = gm.gm_sketch_learned(rp, ids, w, k, 5, params, margin)
        code, st = gm.gm_status(ws)
        assert code == gm.GM_OK
        assert torch.equal(s, s0) and torch.equal(y.view(torch.int64), y0.view(torch.int64))
        T = torch.exp(pred + margin)
        assert st["rows_fallback"] == int((ystar > T.double()).sum()) == len(lens) - 1 - q, q


def test_learned_sketch_arguments():
    X = edge_batch()
    rp, ids, w = gm.to_device(X)
    params = gm.gm_model_init(1)
    L = gm.lib()
    for margin in (float("nan"), float("inf")):
        with pytest.raises(gm.GmError):
            gm.gm_sketch_learned(rp, ids, w, 16, 1, params, margin)
    ws = torch.empty(gm.sketch_learned_workspace_bytes(X.n_rows, X.nnz, 16) - 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(gm.GmError) as e:
        gm.gm_sketch_learned(rp, ids, w, 16, 1, params, 0.0, ws=ws)
    assert e.value.code == gm.GM_ENOMEM
    with pytest.raises(gm.GmError) as e:
        gm.gm_sketch(rp, ids, w, 16, 1, flags=gm.GM_BOUND_LEARNED)
    assert e.value.code == gm.GM_EINVAL
    assert L.gm_model_grad(None, None, None, 0, 0.5, None, None, None, 0, None) == gm.GM_EINVAL


def test_trained_bound_fallback_rate_and_gain():
    tau = 0.9
    ts = learned.make_training_set(12288, ks=(256, 1024, 4096), seed=500)
    params, hist = learned.train(ts, tau=tau, steps=300, log_every=100)
    assert hist[-1][1] < hist[0][1]
    model = learned.BoundModel(params, 0.0, tau)
    # on the information limit: prediction + ln sum v = the tau-quantile of ln max of k Exp(1)
    for k in (256, 1024, 4096):
        rp, ids, w = W.lognormal_batch_device(900 + k, n_rows=512)
        f = gm.gm_features(rp, ids, w, k)
        pred = model.predict(f) + f[:, 1]
        assert abs(float(pred.mean()) - mlp.ystar_quantile(tau, k)) < 0.05, k
    # held-out batch: the learned bound falls back in about 1 - tau of the rows; it
    # keeps fewer arrivals than FastGM without an initial bound (FastSearch's doubling
    # horizon, the method without the network) and about as many as the closed-form
    # quantile, which is the information limit (y* sum v has the same law for every row)
    rp, ids, w = W.lognormal_batch_device(4242, n_rows=4096)
    k = 1024
    s_l, y_l, ws_l = model.sketch(rp, ids, w, k, 3)
    _, st_l = gm.gm_status(ws_l)
    s_c, y_c, ws_c = gm.gm_sketch(rp, ids, w, k, 3)
    _, st_c = gm.gm_status(ws_c)
    s_n, y_n, ws_n = gm.gm_sketch(rp, ids, w, k, 3, flags=gm.GM_BOUND_NONE)
    _, st_n = gm.gm_status(ws_n)
    assert torch.equal(s_l, s_c) and torch.equal(y_l.view(torch.int64), y_c.view(torch.int64))
    assert torch.equal(s_n, s_c) and torch.equal(y_n.view(torch.int64), y_c.view(torch.int64))
    rate = st_l["rows_fallback"] / 4096
    assert abs(rate - (1 - tau)) < 4 * math.sqrt(tau * (1 - tau) / 4096) + 0.02, rate
    assert st_l["kept"] < 0.8 * st_n["kept"]
    assert abs(st_l["kept"] / st_c["kept"] - 1.0) < 0.1
    assert 0.8 < st_l["kept"] / st_c["kept"] < 1.25
