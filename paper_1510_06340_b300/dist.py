"""Host-side helpers for running the solver on several GPUs, one process each.

Events are independent, so ranks exchange no solver data: rank r advances its
own events (global ids r * n .. r * n + n - 1, weak scaling) and the only
collectives are a barrier around the timed region and a max of the elapsed
times.  Works with the gloo (CPU) and nccl backends.
"""
from __future__ import annotations

import os


def world():
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_events(n_per_rank: int, rank: int) -> list[int]:
    """Global event ids owned by `rank` when every rank runs n_per_rank events."""
    return list(range(rank * n_per_rank, (rank + 1) * n_per_rank))


def max_over_ranks(value: float, device=None) -> float:
    """Max of a float over all ranks (identity without an initialised process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()
