"""The multi-rank path on CPU: two gloo ranks shard a batch by rows, sketch their
shards (the CPU oracle stands in for each rank's GPU), and agree on the slowest
rank's time; the shards' sketches are the full batch's rows."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2302_05176_gb300 import dist as D
from paper_2302_05176_gb300 import workloads as W


def test_shard_rows_partition():
    X = W.lognormal_batch(seed=5, n_rows=300, median=200.0)
    for world in (1, 2, 3, 7):
        cuts = [D.shard_rows(X.row_ptr, world, r) for r in range(world)]
        assert cuts[0][0] == 0 and cuts[-1][1] == X.n_rows
        assert all(a[1] == b[0] for a, b in zip(cuts, cuts[1:]))
        work = [int(X.row_ptr[r1] - X.row_ptr[r0]) for r0, r1 in cuts]
        assert max(work) - min(work) <= 2 * int(np.diff(X.row_ptr).max())
    empty = np.zeros(5, dtype=np.int64)
    assert [D.shard_rows(empty, 2, r) for r in range(2)] == [(0, 2), (2, 4)]
    with pytest.raises(ValueError):
        D.shard_rows(X.row_ptr, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, ws, _ = D.env()
    X = W.lognormal_batch(seed=9, n_rows=40, median=60.0)
    r0, r1 = D.shard_rows(X.row_ptr, ws, r)
    rp, ids, w = D.take_rows(X.row_ptr, X.ids, X.w, r0, r1)
    s, y = oracle.sketch(rp, ids, w, 32, 11)
    slowest = D.max_over_ranks(1.0 + r, dist)
    np.savez(os.path.join(out_dir, "rank%d.npz" % r), r0=r0, r1=r1, s=s, y=y, slowest=slowest)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    X = W.lognormal_batch(seed=9, n_rows=40, median=60.0)
    s_full, y_full = oracle.sketch(X.row_ptr, X.ids, X.w, 32, 11)
    covered = 0
    for r in range(2):
        d = np.load(tmp_path / ("rank%d.npz" % r))
        r0, r1 = int(d["r0"]), int(d["r1"])
        assert np.array_equal(d["s"], s_full[r0:r1]) and np.array_equal(d["y"], y_full[r0:r1])
        assert float(d["slowest"]) == 2.0
        covered += r1 - r0
    assert covered == X.n_rows
