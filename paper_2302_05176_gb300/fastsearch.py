"""The paper's own schedule for the first pass (FastSearch, Algorithm 1) on the
GPU, as an ablation of the closed-form and learned bounds.

FastSearch releases, in rounds R = delta, 2 delta, ..., the first
ceil(R v_i / sum v) arrivals of every element until no register of the row is
empty; FastPrune then streams every element up to the row's y*.  The whole
schedule runs in libgm (gm_sketch_fastsearch): one CTA per row runs its rounds on
the FastGM light lanes and warp segments, with no host round trip; this module
only calls it and times it.  The result is gm_sketch's, bit for bit; what
differs is the work: the rounds release arrivals in proportion to the weights
rather than up to a time.
"""
import torch

from . import gm


def fastsearch_sketch(row_ptr, ids, w, k, seed, delta=None, flags=0):
    """Returns (s, y, info): info holds the rounds each row took (int32 tensor), the
    largest of them, the arrivals computed and kept (search and FastPrune
    together) and the GPU time of the call."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    s, y, ws, rounds = gm.gm_sketch_fastsearch(row_ptr, ids, w, k, seed, delta=delta, flags=flags)
    e1.record()
    torch.cuda.synchronize()
    _, st = gm.gm_status(ws)
    info = {"rounds": rounds, "max_rounds": int(rounds.max().item()) if rounds.numel() else 0,
            "arrivals": st["arrivals"], "kept": st["kept"], "ms": e0.elapsed_time(e1)}
    return s, y, info
