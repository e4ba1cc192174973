"""Sharding of the argument arrays over ranks (one process per GPU).

The evaluation has no exchange step: every argument is independent, so rank
r draws and evaluates its own shard (weak scaling) and the only collective is
the benchmark's timing reduction (the slowest rank defines the step time).
"""
from __future__ import annotations


def shard_seed(base_seed: int, rank: int) -> int:
    """Seed of rank r's synthetic shard (distinct per rank, fixed per run)."""
    return base_seed + rank


def shard_range(count: int, rank: int, world: int) -> tuple[int, int]:
    """[lo, hi) of a global array of `count` arguments owned by `rank` when an
    existing array is split instead of drawn per rank (contiguous blocks; the
    first count % world ranks get one extra argument)."""
    base, extra = divmod(count, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of `value` over all ranks of the default process group (or
    the value itself without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
