"""Host logic of the serving engine on a fake device (no GPU): batching by k,
memory-based admission and refusal, malformed requests, cancellation, release,
and shutdown with work queued.  No CUDA call is made."""
import ctypes

import numpy as np
import pytest

from paper_2302_05176_gb300 import gm
from paper_2302_05176_gb300 import server as S


def vec(n, seed=0):
    rng = np.random.default_rng(seed)
    return rng.choice(1 << 24, n, replace=False).astype(np.int32), rng.exponential(size=n)


@pytest.fixture
def srv():
    s = S.Server(device_bytes=64 << 20, fake_device=True, n_streams=2, max_batch_rows=8)
    yield s
    s.close()


def test_requests_finish_and_group_by_k(srv):
    srv.pause()
    tickets = []
    for i in range(20):
        ids, w = vec(100 + i, i)
        tickets.append((srv.submit_sketch(ids, w, 256 if i % 2 else 1024), 256 if i % 2 else 1024))
    assert srv.stats()["queued"] == 20
    srv.pause(False)
    for t, k in tickets:
        rc, res = srv.wait(t, 10.0)
        assert rc == gm.GM_OK and res["k"] == k and 1 <= res["batch_size"] <= 8
        assert res["t_submit_ns"] <= res["t_launch_ns"] <= res["t_done_ns"]
    st = srv.stats()
    assert st["finished"] == 20 and st["sketch_rows"] == 20
    # 10 requests of each k, at most 8 per launch, never mixing k: at least 4 launches
    assert st["sketch_batches"] >= 4
    sizes = {}
    for t, k in tickets:
        sizes.setdefault(k, set()).add(srv.poll(t)[1]["batch_size"])
    assert all(max(v) <= 8 for v in sizes.values())


def test_queries_wait_for_their_sketches(srv):
    srv.pause()
    a = srv.submit_sketch(*vec(50, 1), 64)
    b = srv.submit_sketch(*vec(60, 2), 64)
    j = srv.submit_jaccard(a, b)
    c = srv.submit_cardinality(a)
    assert srv.poll(j)[0] == S.GM_EAGAIN and srv.poll(c)[0] == S.GM_EAGAIN
    srv.pause(False)
    for t in (a, b, j, c):
        assert srv.wait(t, 10.0)[0] == gm.GM_OK
    assert np.isnan(srv.poll(j)[1]["value"])   # the fake device computes nothing
    s, y = srv.read_sketch(a, 64)
    assert (s == -1).all() and np.isinf(y).all()


def test_malformed_requests_are_refused(srv):
    L = S._lib()
    t = ctypes.c_uint64()
    ids, w = vec(10)
    ip, wp = ids.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p)
    assert L.gm_server_submit_sketch(srv._h, ip, wp, 10, 0, ctypes.byref(t)) == gm.GM_EINVAL       # k = 0
    assert L.gm_server_submit_sketch(srv._h, ip, wp, 10, 4097, ctypes.byref(t)) == gm.GM_EINVAL    # k too big
    assert L.gm_server_submit_sketch(srv._h, ip, wp, -1, 64, ctypes.byref(t)) == gm.GM_EINVAL      # nnz < 0
    assert L.gm_server_submit_sketch(srv._h, None, None, 10, 64, ctypes.byref(t)) == gm.GM_EINVAL  # no data
    assert L.gm_server_submit_jaccard(srv._h, 12345, 54321, ctypes.byref(t)) == gm.GM_EINVAL       # unknown
    a = srv.submit_sketch(ids, w, 64)
    b = srv.submit_sketch(ids, w, 128)
    one = srv.submit_sketch(ids, w, 1)
    with pytest.raises(gm.GmError):
        srv.submit_jaccard(a, b)            # different k
    with pytest.raises(gm.GmError):
        srv.submit_cardinality(one)         # k = 1 has no cardinality estimate
    j = srv.submit_cardinality(a)
    with pytest.raises(gm.GmError):
        srv.submit_jaccard(a, j)            # a query is not a sketch
    with pytest.raises(gm.GmError):
        srv.poll(999999)
    assert srv.stats()["submitted"] == 4


def test_admission_refusal_and_resident_memory():
    with S.Server(device_bytes=2 << 20, fake_device=True, n_streams=1) as srv:
        with pytest.raises(gm.GmError) as e:
            srv.submit_sketch(*vec(200_000), 64)     # 2.4 MB of input alone: can never fit
        assert e.value.code == gm.GM_ENOMEM
        assert srv.stats()["refused"] == 1
        # resident sketches of k = 4096 (48 KB each) fill the 2 MB arena until one is refused
        ids, w = vec(1000, 3)
        ts = [srv.submit_sketch(ids, w, 4096) for _ in range(60)]
        rcs = [srv.wait(t, 10.0)[0] for t in ts]
        assert rcs[0] == gm.GM_OK and gm.GM_ENOMEM in rcs
        first_bad = rcs.index(gm.GM_ENOMEM)
        st = srv.stats()
        assert st["arena_resident_bytes"] > (2 << 20) // 2 and st["failed"] >= 1
        # releasing resident sketches makes room again
        for t, rc in zip(ts, rcs):
            if rc == gm.GM_OK:
                srv.release(t)
        assert srv.stats()["arena_resident_bytes"] == 0
        t = srv.submit_sketch(ids, w, 4096)
        assert srv.wait(t, 10.0)[0] == gm.GM_OK
        assert first_bad > 5


def test_cancel_release_and_shutdown():
    srv = S.Server(device_bytes=64 << 20, fake_device=True)
    srv.pause()
    a = srv.submit_sketch(*vec(10, 1), 64)
    b = srv.submit_sketch(*vec(10, 2), 64)
    q = srv.submit_jaccard(a, b)
    assert srv.cancel(a) == gm.GM_OK
    assert srv.poll(a)[0] == S.GM_ECANCELED
    with pytest.raises(gm.GmError):
        srv.submit_cardinality(a)              # a cancelled sketch cannot be queried
    with pytest.raises(gm.GmError) as e:
        srv.release(b)                         # not finished yet
    assert e.value.code == S.GM_EAGAIN
    srv.pause(False)
    assert srv.wait(b, 10.0)[0] == gm.GM_OK
    assert srv.wait(q, 10.0)[0] == gm.GM_EINVAL   # its operand was cancelled
    assert srv.cancel(b) == gm.GM_EINVAL          # already final
    srv.release(b)
    with pytest.raises(gm.GmError):
        srv.release(b)                         # twice
    srv.release(a)                             # a cancelled sketch holds nothing: no-op
    with pytest.raises(gm.GmError):
        srv.read_sketch(b, 64)                 # released
    # shutdown with queued work: it is cancelled, nothing hangs
    srv.pause()
    pending = [srv.submit_sketch(*vec(10, i), 64) for i in range(5)]
    assert srv.stats()["queued"] == 5
    srv.close()
    assert pending


def test_config_validation():
    for kw in ({"n_streams": 0}, {"n_streams": 9}, {"max_batch_rows": 0}, {"device_bytes": 1000},
               {"max_batch_nnz": 1 << 40}):
        with pytest.raises(gm.GmError):
            S.Server(fake_device=True, **kw)
