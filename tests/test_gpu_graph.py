"""gm_sketch captured into a CUDA graph (gm_graph_*): a replay equals the direct
call, and replays read the buffers' current contents (weights rescaled in place,
row boundaries moved)."""
import numpy as np
import pytest
import torch

from paper_2302_05176_gb300 import gm
from paper_2302_05176_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def same(a, b):
    return torch.equal(a[0], b[0]) and torch.equal(a[1].view(torch.int64), b[1].view(torch.int64))


@pytest.mark.parametrize("k", [64, 1024, 4096])  # 4096: the 1024-thread CTA shape
def test_graph_replay_equals_direct_call(k):
    X = W.lognormal_batch(seed=12, n_rows=96, median=900.0)
    rp, ids, w = gm.to_device(X)
    g = gm.SketchGraph(rp, ids, w, k, 5)
    direct = gm.gm_sketch(rp, ids, w, k, 5)[:2]
    out = g.replay()
    torch.cuda.synchronize()
    assert same((out[0].clone(), out[1].clone()), direct)
    # weights doubled in place: registers halve exactly, ids unchanged
    w.mul_(2.0)
    s2, y2 = g.replay()
    torch.cuda.synchronize()
    assert torch.equal(s2, direct[0]) and torch.equal(y2, direct[1] / 2)
    # new row boundaries over the same elements
    cuts = np.sort(np.random.default_rng(1).choice(np.arange(1, X.nnz), size=X.n_rows - 1, replace=False))
    rp.copy_(torch.from_numpy(np.concatenate([[0], cuts, [X.nnz]]).astype(np.int64)))
    out3 = g.replay()
    torch.cuda.synchronize()
    assert same((out3[0].clone(), out3[1].clone()), gm.gm_sketch(rp, ids, w, k, 5)[:2])
    g.close()


def test_graph_create_rejects_bad_arguments():
    X = W.lognormal_batch(seed=13, n_rows=4, median=50.0)
    rp, ids, w = gm.to_device(X)
    with pytest.raises(gm.GmError):
        gm.SketchGraph(rp, ids, w, 0, 1)
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(gm.GmError) as e:
        gm.SketchGraph(rp, ids, w, 64, 1, ws=small)
    assert e.value.code == gm.GM_ENOMEM


def test_tunings_change_work_not_registers():
    """Extreme routings and first-pass quantiles give the registers of the defaults;
    gm_tune returns a valid entry and installs it."""
    X = W.lognormal_batch(seed=14, n_rows=200, median=1500.0)
    rp, ids, w = gm.to_device(X)
    k = 512
    gm.tuning_clear()
    ref = gm.gm_sketch(rp, ids, w, k, 9)[:2]
    mean = X.nnz // X.n_rows
    try:
        for t in ({"light_max": 0.5, "medium_max": 0.5, "heavy_max": 0.5},   # everything dense
                  {"light_max": 1e6, "medium_max": 1e6, "heavy_max": 1e6},   # everything on light lanes
                  {"p_first": 0.9}, {"p_first": 1e-4}):
            gm.tuning_set(k, mean, **t)
            assert same(gm.gm_sketch(rp, ids, w, k, 9)[:2], ref), t
        gm.tuning_clear()
        best, ms = gm.gm_tune(rp, ids, w, k, 9)
        assert ms > 0 and gm.tuning_get(k, mean) == best
        assert same(gm.gm_sketch(rp, ids, w, k, 9)[:2], ref)
    finally:
        gm.tuning_clear()
