"""Multi-GPU sharding of reference locations (host side).

Every location's search is independent (Sec. 2.2): the design is replicated
on each GPU and the reference locations are partitioned, with no collective
on the data path; results are concatenated afterwards (the paper's cluster
runs scatter chunks of locations and gather the outputs the same way,
Sec. 5).  Partitions are contiguous and balanced by a per-location cost
model of the FP32-bulk search.
"""
from __future__ import annotations

import numpy as np


def location_cost(n, Nprime, n0):
    """Relative cost of one location's search: the Schur contraction work
    sum_{j<n} (N' - j) j plus a per-step constant for the FP64 re-score and
    update (in units of one candidate-coordinate FMA)."""
    n = np.asarray(n, dtype=np.float64)
    Np = np.asarray(Nprime, dtype=np.float64)
    # sum_{j=0}^{n-1} (Np - j) j = Np n(n-1)/2 - (n-1)n(2n-1)/6
    contraction = Np * n * (n - 1) / 2 - (n - 1) * n * (2 * n - 1) / 6
    return contraction + 2000.0 * n + Np


def partition(cost, world_size):
    """Contiguous [start, end) ranges, one per rank, with near-equal total cost."""
    cost = np.asarray(cost, dtype=np.float64)
    M = len(cost)
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    cum = np.concatenate([[0.0], np.cumsum(cost)])
    total = cum[-1]
    bounds = [0]
    for r in range(1, world_size):
        b = int(np.searchsorted(cum, total * r / world_size, side="left"))
        bounds.append(min(max(b, bounds[-1]), M))
    bounds.append(M)
    return [(bounds[r], bounds[r + 1]) for r in range(world_size)]


def run_sharded(compute, Xref, n, Nprime, n0, rank, world_size, group=None):
    """Compute this rank's share of the locations with `compute(lo, hi)`
    (returning a dict of 1-d numpy arrays over [lo, hi)), then gather every
    rank's share so that each rank ends with the full, ordered result.
    Collectives: one all_gather_object of the per-rank outputs."""
    import torch.distributed as dist

    M = len(Xref)
    ranges = partition(location_cost(np.broadcast_to(n, (M,)), np.broadcast_to(Nprime, (M,)), n0),
                       world_size)
    lo, hi = ranges[rank]
    mine = compute(lo, hi)
    parts = [None] * world_size
    if world_size > 1:
        dist.all_gather_object(parts, (lo, hi, mine), group=group)
    else:
        parts = [(lo, hi, mine)]
    parts.sort(key=lambda t: t[0])
    keys = mine.keys()
    return {k: np.concatenate([p[2][k] for p in parts]) for k in keys}
