"""gm_sketch_host: a CSR batch in host memory, pipelined in row chunks over two
streams, gives gm_sketch's registers -- pinned and pageable buffers, batches of
one chunk and of several, empty rows; bad row offsets are refused on the host."""
import numpy as np
import pytest
import torch

from paper_2302_05176_gb300 import gm
from paper_2302_05176_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_rows,k,pinned", [(300, 64, False), (3000, 256, True), (5000, 1024, True)])
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
