"""Stream-FastGM on the GPU (gm_stream_*): a stream with repeated elements folded
chunk by chunk equals the sketch of its distinct set -- bit for bit against
gm_sketch of that set, and within the parity tolerance against the oracle's
Algorithm 2 run over the same stream -- for any chunking, including empty
chunks, chunks of repeats and chunks long enough to be split across CTAs."""
import numpy as np
import pytest
import torch

import oracle
from paper_2302_05176_gb300 import gm
from paper_2302_05176_gb300 import workloads as W
from parity import compare_sketch

pytestmark = pytest.mark.gpu
SEED = 31


def distinct_set(n, seed):
    rng = np.random.default_rng(seed)
    ids = rng.choice(1 << 24, n, replace=False).astype(np.int32)
    w = W.pareto_weights(rng, n, 1.2, 1e-3)
    return ids, w


def occurrence_stream(ids, w, seed, max_rep=4):
    rng = np.random.default_rng(seed)
    rep = rng.integers(1, max_rep + 1, size=ids.size)
    order = rng.permutation(np.repeat(np.arange(ids.size), rep))
    return ids[order], w[order]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("k", [64, 1024, 4096])
def test_stream_equals_distinct_set(k):
    ids, w = distinct_set(30000, k)
    sid, sw = occurrence_stream(ids, w, k + 1)
    rp = torch.tensor([0, ids.size], dtype=torch.int64, device="cuda")
    s_ref, y_ref, _ = gm.gm_sketch(rp, dev(ids), dev(w), k, SEED)
    cuts = [0, 1, 8, 1008, 1008, 41008, sid.size]  # a single element, an empty chunk, a chunk > 32768
    st = gm.StreamSketch(k, SEED)
    for a, b in zip(cuts, cuts[1:]):
        st.ingest(dev(sid[a:b]), dev(sw[a:b]))
    assert torch.equal(st.s, s_ref[0]) and torch.equal(st.y.view(torch.int64), y_ref[0].view(torch.int64))
    # the oracle's Algorithm 2 over the same stream (host, FP64)
    s_o, y_o, _ = oracle.stream_fastgm(sid, sw, k, SEED)
    s_f, y_f, y2, s2 = oracle.sketch(np.array([0, ids.size]), ids, w, k, SEED, runner_up=True)
    assert np.array_equal(s_f[0], s_o) and np.array_equal(y_f[0], y_o)  # Algorithm 2 = the unpruned stream
    rep = compare_sketch(st.s.cpu().numpy()[None], st.y.cpu().numpy()[None], s_o[None], y_o[None], y2, s2)
    assert rep["ok"], rep


def test_repeats_and_empty_chunks_change_nothing():
    k = 256
    ids, w = distinct_set(5000, 3)
    st = gm.StreamSketch(k, SEED)
    st.ingest(dev(ids), dev(w))
    s0, y0 = st.s.clone(), st.y.clone()
    st.ingest(dev(ids[::-1].copy()), dev(w[::-1].copy()))   # all repeats
    st.ingest(dev(ids[:0]), dev(w[:0]))                       # empty
    assert torch.equal(st.s, s0) and torch.equal(st.y.view(torch.int64), y0.view(torch.int64))


def test_later_chunks_are_mostly_screened():
    """Once the running sketch is full, a chunk of fresh elements of similar weight
    is bounded by y*: almost every element fails the first-arrival screen."""
    k = 1024
    ids, w = distinct_set(400000, 9)
    w = np.random.default_rng(2).exponential(size=ids.size)
    st = gm.StreamSketch(k, SEED)
    st.ingest(dev(ids[:200000]), dev(w[:200000]))
    st.ingest(dev(ids[200000:]), dev(w[200000:]))
    code, stats = gm.gm_status(st.ws)
    assert code == gm.GM_OK
    assert stats["screened_out"] > 0.9 * 200000, stats
    assert stats["kept"] < 20 * k, stats
