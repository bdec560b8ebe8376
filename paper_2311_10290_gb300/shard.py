"""Splitting one estimate over processes (one per GPU) and merging it.

Samples are independent and every quantity the estimators of Alg. 2 and
Alg. 4 use is an integer sum over samples (visits per node, uniform-walk
passes per node, sum Y1, sum Y2).  Process r of W therefore draws a disjoint,
contiguous range of sample ids (set with LAP_OPT_CURSOR before its first
lap_sample) and the totals are one element-wise sum: a single all-reduce of
the uint64 counts (16 n + 24 bytes), after which any handle finalizes them
(lap_set_counts, then lap_ecc / lap_kemeny) exactly as if it had drawn every
sample.  Host-side logic only: the sampling itself runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np


def id_range(rank: int, world: int, total: int, first: int = 0):
    """(first id, count) of process `rank` when `total` sample ids starting at
    `first` are split into `world` contiguous ranges whose sizes differ by at
    most one (lower ranks take the extra ids)."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad rank/world/total")
    base, extra = divmod(int(total), int(world))
    start = first + rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def allreduce_counts(cnt1, cnt2, sums, group=None):
    """Sums (cnt1[n], cnt2[n], sums[3] = {omega, sum Y1, sum Y2}) over the
    processes of `group` in place.  Accepts torch int64 tensors (uint64
    counts reinterpreted: the sum modulo 2^64 is the same) or numpy uint64
    arrays (copied through a CPU tensor); returns the three totals."""
    import torch
    import torch.distributed as dist

    def as_tensor(a):
        if isinstance(a, torch.Tensor):
            return a, False
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64).copy()), True

    out = []
    for a in (cnt1, cnt2, sums):
        t, converted = as_tensor(a)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        out.append(t.numpy().view(np.uint64) if converted else t)
    return tuple(out)
