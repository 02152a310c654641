"""Host-side logic for running the ray trace on several ranks.

Sources are independent (the paper's MPI mode, Sec. 3.2-3.3): each rank traces a
subset and the rate fields are summed.  Subsets are balanced by work, which is
proportional to the traced volume (4/3) pi R^3 of each source (Sec. 4.2), with
the longest-processing-time-first rule.  The sum of the rate fields is the one
exchange step; every box of the pool this library is built on has a single GPU,
so the collective is exercised with CPU (gloo) process groups.
"""
from __future__ import annotations

import heapq

import numpy as np


def lpt_shards(radius, world):
    """Rank of every source: longest first, each to the least loaded rank."""
    work = (4.0 / 3.0) * np.pi * np.asarray(radius, dtype=np.float64) ** 3
    order = np.argsort(-work, kind="stable")
    heap = [(0.0, r) for r in range(world)]
    owner = np.empty(len(work), dtype=np.int64)
    for i in order:
        load, r = heapq.heappop(heap)
        owner[i] = r
        heapq.heappush(heap, (load + work[i], r))
    return owner


def shard_loads(radius, owner, world):
    work = (4.0 / 3.0) * np.pi * np.asarray(radius, dtype=np.float64) ** 3
    return np.bincount(owner, weights=work, minlength=world)


def sum_rates(gamma, dist, group=None):
    """Sum the ranks' partial rate fields in place (all ranks get the total)."""
    dist.all_reduce(gamma, op=dist.ReduceOp.SUM, group=group)
    return gamma


def aggregate(ms_local, units_local, dist, device=None):
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms = float(t.item())
    return ms, float(u.item()) / (ms * 1e-3)


def shard(pos, ndot, radius, rank, world):
    """This rank's share of a source catalogue (the whole catalogue for world == 1)."""
    if world <= 1:
        return pos, ndot, radius
    mine = lpt_shards(radius, world) == rank
    return pos[mine], ndot[mine], radius[mine]


class ShardedStep:
    """One step of the sharded forward path on one rank: trace this rank's
    sources into the rate field, sum the partial fields over the ranks (the
    exchange step), then run the elementwise chemistry on the full field
    (replicated on every rank).  ``trace(gamma)`` and ``chemistry(gamma)`` are
    callables that fill / consume the rank's field; with one rank the sum is
    skipped."""

    def __init__(self, trace, chemistry, dist=None, world=1, group=None):
        self.trace = trace
        self.chemistry = chemistry
        self.dist = dist
        self.world = world
        self.group = group

    def __call__(self, gamma):
        self.trace(gamma)
        if self.world > 1:
            sum_rates(gamma, self.dist, self.group)
        return self.chemistry(gamma)
