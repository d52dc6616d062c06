"""Sharding of independent instances over ranks (one process per GPU).

Instances never interact, so a multi-GPU run needs no collective on the data
path: each rank integrates its own instances and only the timing is reduced.
Weak scaling gives every rank a full workload of its own (seeded by rank);
strong scaling splits one workload into contiguous, near-equal shards.
"""
from __future__ import annotations


def shard_bounds(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [lo, hi) of n instances owned by `rank` out of `world` (sizes differ by at most 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    base, extra = divmod(int(n), int(world))
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s own workload under weak scaling."""
    return int(base_seed) + 1000 * int(rank)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Largest `value` over all ranks (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
