"""gm_sketch_noalloc: the entry point for callers that cannot allocate device memory.

Some callers cannot give the library a workspace (their device memory belongs
to a framework allocator, or they must never stall on cudaMalloc, or their
binding can only pass input and output buffers).  gm_sketch_noalloc keeps its
scratch in a fixed device array inside libgm instead.  This test calls it through
the C-ABI several times in a row on different inputs -- including a row longer
than 32,768 elements at k = 4096, which uses the array's long-row regions and the
1024-thread kernels -- and checks each result against gm_sketch on the same
input, within the tolerance the other GPU tests use, and the array's device
status through gm_sketch_noalloc_status.  It builds its own inputs so it passes
alone in a fresh process as well as after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2302_05176_gb300 import build as libbuild
from paper_2302_05176_gb300 import gm
from paper_2302_05176_gb300 import workloads as W
from parity import compare_sketch

pytestmark = pytest.mark.gpu

GM_NOALLOC_MAX_NNZ = 1 << 20
GM_NOALLOC_MAX_ROWS = 1 << 16


@pytest.fixture(scope="module")
def noalloc():
    lib = ctypes.CDLL(libbuild.build())
    f = lib.gm_sketch_noalloc
    vp = ctypes.c_void_p
    f.argtypes = [vp, vp, vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32,
                  vp, vp, vp]
    f.restype = ctypes.c_int
    return f


@pytest.fixture(scope="module")
def noalloc_status():
    lib = ctypes.CDLL(libbuild.build())
    f = lib.gm_sketch_noalloc_status
    f.argtypes = [ctypes.POINTER(gm.gm_stats), ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _run_noalloc(fn, X, k, seed, flags=0):
    rp, ids, w = gm.to_device(X)
    s = torch.full((X.n_rows, k), -7, dtype=torch.int32, device="cuda")
    y = torch.full((X.n_rows, k), -7.0, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(_p(rp), _p(ids), _p(w), X.n_rows, X.nnz, k, seed, flags, _p(s), _p(y), stream)
    assert rc == 0, gm.strerror(rc)
    torch.cuda.synchronize()
    return s.cpu().numpy(), y.cpu().numpy()


def _run_reference(X, k, seed):
    rp, ids, w = gm.to_device(X)
    s, y, ws = gm.gm_sketch(rp, ids, w, k, seed)
    assert gm.gm_status(ws)[0] == gm.GM_OK
    return s.cpu().numpy(), y.cpu().numpy()


def test_noalloc_matches_gm_sketch_twice(noalloc, noalloc_status):
    torch.cuda.set_device(0)
    rng = np.random.default_rng(23)
    long_row = [(np.sort(rng.choice(1 << 24, size=n, replace=False)).astype(np.int32),
                 W.pareto_weights(rng, n, 1.2, 1e-3)) for n in (100_000, 3, 1500)]
    # the last call compacts its long row (GM_FLAG_COMPACT_LONG: the row's survivor
    # lists and unit counts live in the same scratch)
    cases = [(W.lognormal_batch(seed=21, n_rows=48, median=500.0, hi=6000), 1024, 7, 0),
             (W.uniform_rows(seed=22, n_rows=9, n_pos=[0, 1, 40, 300, 2500, 7, 64, 1000, 3]), 256, 8, 0),
             (W.from_rows(long_row), 4096, 9, 0),
             (W.from_rows(long_row), 4096, 9, gm.GM_FLAG_COMPACT_LONG)]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for X, k, seed, flags in cases:  # calls in a row through the shared scratch
        s, y = _run_noalloc(noalloc, X, k, seed, flags)
        st = gm.gm_stats()
        assert noalloc_status(ctypes.byref(st), stream) == gm.GM_OK
        # the counters are this call's: every positive element visited at least once
        # (a row redone with a wider bound visits its elements again)
        assert st.status == gm.GM_OK and st.elements >= int(np.count_nonzero(X.w > 0)) > 0
        s_ref, y_ref = _run_reference(X, k, seed)
        rep = compare_sketch(s, y, s_ref, y_ref)
        assert rep["ok"], rep
        assert np.array_equal(s, s_ref)  # same kernels: identical registers


def test_noalloc_rejects_inputs_beyond_its_scratch(noalloc):
    # rejected on the host before any launch, so the pointers are never touched
    fake = ctypes.c_void_p(0x1000)
    rc = noalloc(fake, fake, fake, 1, GM_NOALLOC_MAX_NNZ + 1, 64, 1, 0, fake, fake, None)
    assert rc == gm.GM_ENOMEM
    rc = noalloc(fake, fake, fake, 2 * GM_NOALLOC_MAX_ROWS, 100, 64, 1, 0, fake, fake, None)
    assert rc == gm.GM_ENOMEM
    rc = noalloc(fake, fake, fake, 1, 10, gm.GM_MAX_K + 1, 1, 0, fake, fake, None)
    assert rc == gm.GM_EINVAL
