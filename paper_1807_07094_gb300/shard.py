"""Source sharding of the tracer over ranks (one GPU per rank).

The rates of disjoint source sets add: each source's rays deposit into the
cells independently of every other source's (Sec. 2.1 step iii traces the
sources one after another into the same rate fields; Eq. ion is linear in the
photons).  So every rank holds the whole gas field, traces its own subset of
the sources into its own rate fields, and one SUM all-reduce of the six rate
fields and of the photon-budget terms gives every rank the totals that the
chemistry needs (the paper's version-1 decomposition, Sec. 2.1, with the MPI
sum of step C3).

Nothing here computes: the partition is host bookkeeping and the reduction
is one torch.distributed collective over tensors the tracer filled.
"""
from __future__ import annotations

from typing import List

import numpy as np


def partition_sources(ndot, world: int) -> List[np.ndarray]:
    """Indices of the sources each of `world` ranks traces.

    Sources are dealt brightest first to the rank with the least luminosity so
    far (longest-processing-time greedy): a source's ray tree, and so its
    tracing work, grows with its luminosity.  Every source goes to exactly one
    rank; each rank's list is in ascending index order."""
    ndot = np.asarray(ndot, np.float64)
    tot = ndot.reshape(ndot.shape[0], -1).sum(axis=1)
    order = np.argsort(-tot, kind="stable")
    load = np.zeros(world)
    parts = [[] for _ in range(world)]
    for i in order:
        r = int(np.argmin(load))
        parts[r].append(int(i))
        load[r] += tot[i]
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def allreduce_rates(gamma, heat, budget=None, group=None):
    """SUM all-reduce, in place, of a rank's rate fields (torch tensors [3, n,
    n, n]) and, if given, of its photon budget (launched, absorbed, escaped,
    emitted; returned summed as a numpy array)."""
    import torch
    import torch.distributed as dist
    dist.all_reduce(gamma, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(heat, op=dist.ReduceOp.SUM, group=group)
    if budget is None:
        return None
    dev = gamma.device
    b = torch.tensor(np.asarray(budget, np.float64), dtype=torch.float64, device=dev)
    dist.all_reduce(b, op=dist.ReduceOp.SUM, group=group)
    return b.cpu().numpy()
