"""Sharding of one chemistry step over ranks (one process per GPU).

Every cell, and every box, is advanced independently within a step, so the step shards with no
exchange: each rank advances its own share and the only collectives are a gather of the results
(when one rank needs the whole field) and a max-reduction of the step time.  Shares are balanced
by predicted cost, e.g. the substep counts the previous step left (1 for a bulk-accepted cell,
1 + implicit substeps for a stiff one), with the greedy longest-processing-time rule.
"""
import numpy as np


def partition_by_cost(cost, world):
    """Indices of the units (cells or boxes) of each rank: units sorted by decreasing cost, each
    given to the rank with the smallest load so far (ties to the lower rank); every rank's indices
    are returned in increasing order.  Deterministic, so every rank computes the same partition."""
    cost = np.asarray(cost, dtype=np.float64)
    if world < 1:
        raise ValueError("world must be >= 1")
    order = np.argsort(-cost, kind="stable")
    load = np.zeros(world)
    owner = np.empty(cost.size, dtype=np.int64)
    for u in order:
        r = int(np.argmin(load))
        owner[u] = r
        load[r] += cost[u]
    return [np.nonzero(owner == r)[0] for r in range(world)]


def max_over_ranks(value, dist=None):
    """The maximum of a per-rank scalar (e.g. a step time) over all ranks."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_field(local, parts, n_total, dist=None, dst=0):
    """Reassemble per-rank results into the whole field on rank `dst`.  local: [m_r, ...] array of
    this rank's units in the order of parts[rank]; returns the [n_total, ...] array on dst (None
    elsewhere)."""
    local = np.ascontiguousarray(local)
    if dist is None:
        out = np.empty((n_total,) + local.shape[1:], dtype=local.dtype)
        out[parts[0]] = local
        return out
    rank, world = dist.get_rank(), dist.get_world_size()
    gathered = [None] * world if rank == dst else None
    dist.gather_object(local, gathered, dst=dst)
    if rank != dst:
        return None
    out = np.empty((n_total,) + local.shape[1:], dtype=local.dtype)
    for r in range(world):
        out[parts[r]] = gathered[r]
    return out
