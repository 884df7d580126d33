"""Scenario sharding across ranks (one process per GPU).

N-1 scenarios are independent, so a screen shards its outage list across
ranks with no collective on the data path; only results are gathered, and
for the adjoint the gradient sums are all-reduced once at the end.  These
helpers are the host side of that: they work with any torch.distributed
backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import numpy as np


def shard_bounds(S: int, rank: int, world: int):
    """Contiguous [lo, hi) slice of S scenarios for `rank` (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(S, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def shard_outages(outages, rank: int, world: int):
    lo, hi = shard_bounds(len(outages), rank, world)
    return np.asarray(outages)[lo:hi]


def _dist():
    import torch.distributed as dist
    return dist


def max_over_ranks(value: float, device=None) -> float:
    """Max of a scalar over all ranks (1 when not distributed)."""
    dist = _dist()
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(a: np.ndarray, device=None) -> np.ndarray:
    """Elementwise sum of an FP64 array over ranks (the adjoint's gradients)."""
    dist = _dist()
    if not (dist.is_available() and dist.is_initialized()):
        return np.asarray(a, dtype=np.float64)
    import torch
    t = torch.as_tensor(np.asarray(a, dtype=np.float64), device=device).clone()
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy()


def gather_rows(a: np.ndarray, S: int, device=None):
    """Rank 0 receives the full [S, ...] array assembled from every rank's
    contiguous shard (shard_bounds); other ranks receive None."""
    dist = _dist()
    if not (dist.is_available() and dist.is_initialized()):
        return np.asarray(a)
    import torch
    rank, world = dist.get_rank(), dist.get_world_size()
    a = np.asarray(a)
    tail = a.shape[1:]
    width = max(shard_bounds(S, r, world)[1] - shard_bounds(S, r, world)[0] for r in range(world))
    buf = np.zeros((width,) + tail, dtype=a.dtype)
    buf[:a.shape[0]] = a
    t = torch.as_tensor(buf, device=device)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t)
    if rank != 0:
        return None
    out = [p.cpu().numpy()[:shard_bounds(S, r, world)[1] - shard_bounds(S, r, world)[0]]
           for r, p in enumerate(parts)]
    return np.concatenate(out, axis=0)
