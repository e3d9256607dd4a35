"""The paper's own schedule for the first pass (FastSearch, Algorithm 1) on the
GPU, as an ablation of the closed-form and learned bounds.

FastSearch releases, in rounds R = delta, 2 delta, ..., the first
ceil(R v_i / sum v) arrivals of every element until no register of the row is
empty; FastPrune then streams every element up to the row's y*.  On the GPU a
round is one gm_sketch_budget launch over the rows not yet filled (rows already
filled keep their budget, so their registers come out the same again), and
FastPrune is gm_sketch_bounded with the per-row y* of the last round as the exact
bound.  The result is gm_sketch's, bit for bit; what differs is the work: the
rounds release arrivals in proportion to the weights rather than up to a time.
"""
import time

import torch

from . import gm


def fastsearch_sketch(row_ptr, ids, w, k, seed, delta=None, max_rounds=100000, flags=0):
    """Returns (s, y, info): info holds the rounds, the per-row final budget R, the
    arrivals released by the budgets that filled each row (FastSearch's work), and
    FastPrune's kept arrivals and the GPU time of each phase."""
    n_rows, nnz = row_ptr.numel() - 1, ids.numel()
    dev = row_ptr.device
    delta = int(delta or k)
    R = torch.zeros(n_rows, dtype=torch.float64, device=dev)
    # rows without a positive weight never fill: they are done from the start
    row_of = torch.repeat_interleave(torch.arange(n_rows, device=dev), row_ptr[1:] - row_ptr[:-1],
                                     output_size=nnz)
    pos = torch.zeros(n_rows, dtype=torch.int64, device=dev).index_add_(0, row_of, (w > 0).to(torch.int64))
    done = pos == 0
    s = torch.empty((n_rows, k), dtype=torch.int32, device=dev)
    y = torch.empty((n_rows, k), dtype=torch.float64, device=dev)
    ws = gm.workspace(n_rows, nnz, k)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    rounds = 0
    ystar = None
    while rounds < max_rounds:
        rounds += 1
        R[~done] = float(rounds * delta)
        gm.gm_sketch_budget(row_ptr, ids, w, k, seed, R, flags=flags, s_out=s, y_out=y, ws=ws)
        ystar = gm.gm_row_ystar(y)
        done |= torch.isfinite(ystar)
        if bool(done.all()):
            break
    e1.record()
    _, st_search = gm.gm_status(ws)
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    bound = torch.where(torch.isfinite(ystar), ystar, torch.full_like(ystar, -1.0))  # -1: closed form
    e2.record()
    s2, y2, ws2 = gm.gm_sketch_bounded(row_ptr, ids, w, k, seed, bound, flags=flags)
    e3.record()
    torch.cuda.synchronize()
    _, st_prune = gm.gm_status(ws2)
    info = {"rounds": rounds, "R": R, "search_arrivals": st_search["arrivals"], "prune_kept": st_prune["kept"],
            "prune_arrivals": st_prune["arrivals"], "search_ms": e0.elapsed_time(e1),
            "prune_ms": e2.elapsed_time(e3)}
    return s2, y2, info
