"""Host-side logic for running on several GPUs of one node (one process per GPU).

The rt-BTE right-hand side shards two ways:

* independent instances (an ensemble of simulations, or replicas of one workload): each
  rank integrates its own instances and no data crosses ranks; whole-job throughput is the
  units all ranks processed over the slowest rank's time (weak scaling);
* destination rows of one instance (the collision integral of a row reads the whole
  population vector but writes only its own row, Eq. e-ph and Eq. ph-ph): each rank owns a
  contiguous slice of rows balanced by stored channel entries, evaluates them, and the
  slices are all-gathered once per stage; the WRMS error norm is a sum of squares, so one
  scalar all-reduce per attempt gives the global norm.

This module holds the partitioning and reduction arithmetic shared by bench.py and the
tests.  The row split runs through the library: a rank counts every row's channels
(Context.upload_channels(count_only=True), Context.row_entries), takes its slice from
balanced_slices, and creates a Context with row_range=(begin, end), which stores and streams
only that slice's channels; rtbte_rhs then fills the slice's rows and writes 0 elsewhere.
"""
from __future__ import annotations

import numpy as np


def balanced_slices(weights, world: int) -> list[tuple[int, int]]:
    """Contiguous [begin, end) slices of len(weights) items, one per rank, with prefix sums of
    the weights split as evenly as the item boundaries allow (ties to the earlier item)."""
    w = np.asarray(weights, dtype=np.float64)
    if world < 1:
        raise ValueError("world must be >= 1")
    pre = np.concatenate([[0.0], np.cumsum(w)])
    total = pre[-1]
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        cuts.append(max(cuts[-1], int(np.searchsorted(pre, target, side="left"))))
    cuts.append(len(w))
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def instance_shards(weights, world: int) -> list[list[int]]:
    """Instances per rank for an ensemble: largest first onto the least-loaded rank (LPT), each
    rank's list in ascending instance order.  Every instance appears exactly once."""
    w = np.asarray(weights, dtype=np.float64)
    load = np.zeros(world)
    out: list[list[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(w)), key=lambda k: (-w[k], k)):
        r = int(np.argmin(load))
        out[r].append(i)
        load[r] += w[i]
    return [sorted(x) for x in out]


def job_throughput(units: float, ms: float, dist=None, device=None) -> tuple[float, float]:
    """(units summed over ranks, max over ranks of ms): whole-job rate = units / max ms.
    With dist=None (one process) the local values are returned."""
    if dist is None:
        return float(units), float(ms)
    import torch

    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(u)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())
