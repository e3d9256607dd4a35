"""Multi-rank helpers: one process per GPU, rows sharded with no collective on
the data path (rows are independent sketches).  Only the timing uses a
collective (the maximum over ranks).  Works with the nccl backend on GPUs and
with gloo on CPU."""
import os

import numpy as np


def env():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def shard_rows(row_ptr, world, rank):
    """Contiguous row range [r0, r1) of `rank`, cut where the cumulative element
    count crosses rank/world of the total, so shards hold near-equal work."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    n_rows = row_ptr.size - 1
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    nnz = int(row_ptr[-1])

    def cut(j):
        if j <= 0:
            return 0
        if j >= world:
            return n_rows
        if nnz == 0:
            return n_rows * j // world
        return int(np.searchsorted(row_ptr[1:], nnz * j / world, side="left")) + 1

    r0, r1 = cut(rank), cut(rank + 1)
    return min(r0, r1), r1


def take_rows(row_ptr, ids, w, r0, r1):
    """The CSR of rows [r0, r1) (row_ptr rebased to 0)."""
    lo, hi = int(row_ptr[r0]), int(row_ptr[r1])
    return np.asarray(row_ptr[r0:r1 + 1]) - lo, ids[lo:hi], w[lo:hi]


def max_over_ranks(x, dist=None, device="cpu"):
    """The maximum of a float over all ranks (x itself without a process group)."""
    if dist is None or not dist.is_initialized():
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
