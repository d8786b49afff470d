"""Rank-level helpers for running on several GPUs (one process per GPU).

Batches of independent problems split across ranks without any data-path
collective (each rank owns whole problems); timings are combined with a
max-reduction over ranks.  Host-side logic only: it is covered by multi-process
CPU tests with the gloo backend.
"""
from __future__ import annotations


def shard_problems(sizes, rank: int, world: int) -> list[int]:
    """Indices of the problems rank `rank` owns out of `world` ranks.

    Greedy longest-processing-time assignment on the problem sizes (grid points,
    i.e. work per step): every problem goes to exactly one rank and the largest
    per-rank load is within one problem of the mean.  Deterministic: ties are
    broken by problem index and by rank.
    """
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    load = [0] * world
    owner = [0] * len(sizes)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += int(sizes[i])
    return [i for i in range(len(sizes)) if owner[i] == rank]


def max_over_ranks(values, dist=None, device=None) -> list[float]:
    """Element-wise maximum of a list of floats over all ranks (identity on one rank)."""
    vals = [float(v) for v in values]
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return vals
    import torch

    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def sum_over_ranks(values, dist=None, device=None) -> list[float]:
    vals = [float(v) for v in values]
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return vals
    import torch

    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [float(x) for x in t.tolist()]
