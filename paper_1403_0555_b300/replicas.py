"""Replicas across GPUs, for weak scaling.

The enumeration shards with no exchange: starts and orbits are independent.
So with N GPUs every rank runs the same workload shape on orbits of its own
seeds. The only cross-rank step is the timing reduction. Throughput is all
ranks' converged copies over the slowest rank's time.

These are the host pieces of that, kept apart from the GPU code so that they
run, and are tested, on CPU ranks with the gloo backend.
"""
from __future__ import annotations


def rank_seed(rank: int, j: int) -> int:
    """Seed and orbit id of orbit j on `rank`.  Rank 0 keeps the single-GPU
    workload's seeds (j + 1); rank r draws its own from 1000 r + j + 1."""
    return 1000 * rank + j + 1


def reduce_timing(dist, ms: float, count: float, device=None):
    """(max over ranks of ms, sum over ranks of count); `dist` is
    torch.distributed with an initialised process group, or None on one GPU."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms), float(count)
    import torch
    t = torch.tensor([float(ms), float(count)], dtype=torch.float64, device=device)
    m = t.clone()
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(m[0]), float(t[1])
