"""Independent replicas across ranks (one process per GPU).

The instances of this hot path do not exchange data: with N ranks, each rank
runs its own instance of the workload with its own seed, and there is no
collective on the data path. The only cross-rank step is the timing
reduction: the slowest rank's time, and the throughput of all ranks'
particle-steps over that time.
"""
from __future__ import annotations


def rank_seed(seed: int, rank: int) -> int:
    """Seed of a rank's instance: independent replicas of the same workload."""
    return int(seed) + int(rank)


def max_over_ranks(values, dist=None, device=None):
    """Element-wise maximum of `values` over all ranks (the values unchanged
    with one process)."""
    vals = [float(v) for v in values]
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return vals
    import torch
    t = torch.tensor(vals, dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def throughput(n_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Particle-steps per second of the whole job: all ranks' work over the
    slowest rank's time."""
    return float(n_per_rank) * float(steps) * float(world) / float(seconds)
