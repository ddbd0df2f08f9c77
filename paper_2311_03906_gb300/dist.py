"""Host-side multi-rank helpers: one process per GPU, each sampling its own
shot range (records depend only on (seed, global shot index), so ranks need
no data exchange), and the max-over-ranks timing used for weak scaling."""
from __future__ import annotations

import os
from typing import Tuple


def world() -> Tuple[int, int, int]:
    """(world size, rank, local rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_range(rank: int, world_size: int, shots_per_rank: int, step: int, steps_total: int) -> Tuple[int, int]:
    """Global shot range [start, start + shots_per_rank) of `rank` at `step`.
    Ranks own disjoint blocks of steps_total * shots_per_rank shots, so every
    (rank, step) pair samples distinct shots."""
    if not 0 <= rank < world_size or not 0 <= step < steps_total:
        raise ValueError("rank or step out of range")
    start = (rank * steps_total + step) * shots_per_rank
    return start, start + shots_per_rank


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
