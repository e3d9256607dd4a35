"""gm_sketch_host: a CSR batch in host memory, pipelined in row chunks over eight
streams, gives gm_sketch's registers -- pinned and pageable buffers, batches of
one chunk and of several (more chunks than streams), empty rows, chunks of very
unequal size; the workspace is sized by the largest chunk; bad row offsets are
refused on the host."""
import numpy as np
import pytest
import torch

from paper_2302_05176_gb300 import gm
from paper_2302_05176_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_rows,k,pinned", [(300, 64, False), (3000, 256, True), (5000, 1024, True),
                                              (600, 4096, True)])
def test_host_pipeline_equals_device_call(n_rows, k, pinned):
    X = W.lognormal_batch(seed=n_rows, n_rows=n_rows, median=400.0)
    X.w[X.row_ptr[7]:X.row_ptr[8]] = 0.0  # a row without positive weights
    rp, ids, w = (torch.from_numpy(a) for a in (X.row_ptr, X.ids, X.w))
    if pinned:
        rp, ids, w = rp.pin_memory(), ids.pin_memory(), w.pin_memory()
    s, y, _ = gm.gm_sketch_host(rp, ids, w, k, 5)
    s0, y0, _ = gm.gm_sketch(*gm.to_device(X), k, 5)
    assert torch.equal(s, s0.cpu()) and torch.equal(y.view(torch.int64), y0.cpu().view(torch.int64))


def test_host_pipeline_refuses_bad_offsets():
    X = W.lognormal_batch(seed=2, n_rows=20, median=50.0)
    rp = torch.from_numpy(X.row_ptr.copy())
    ids, w = torch.from_numpy(X.ids), torch.from_numpy(X.w)
    rp[5], rp[6] = rp[6].item(), rp[5].item()  # decreasing
    with pytest.raises(gm.GmError) as e:
        gm.gm_sketch_host(rp, ids, w, 64, 1)
    assert e.value.code == gm.GM_EINVAL


def test_host_workspace_sized_by_the_largest_chunk():
    rng = np.random.default_rng(4)
    lens = np.where(np.arange(3000) < 150, 3000, rng.integers(0, 6, 3000))  # the first chunk holds most elements
    rows = [(rng.choice(1 << 24, int(n), replace=False).astype(np.int32), rng.exponential(size=int(n))) for n in lens]
    X = W.from_rows(rows)
    rp, ids, w = (torch.from_numpy(a) for a in (X.row_ptr, X.ids, X.w))
    k = 128
    L = gm.lib()
    tight = L.gm_sketch_host_workspace_bytes_csr(gm._ptr(rp), X.n_rows, k)
    loose = L.gm_sketch_host_workspace_bytes(X.n_rows, X.nnz, k)
    assert 0 < tight <= loose
    short = torch.empty(tight - 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(gm.GmError) as e:
        gm.gm_sketch_host(rp, ids, w, k, 9, ws=short)
    assert e.value.code == gm.GM_ENOMEM
    s, y, _ = gm.gm_sketch_host(rp, ids, w, k, 9)
    s0, y0, _ = gm.gm_sketch(*gm.to_device(X), k, 9)
    assert torch.equal(s, s0.cpu()) and torch.equal(y.view(torch.int64), y0.cpu().view(torch.int64))
