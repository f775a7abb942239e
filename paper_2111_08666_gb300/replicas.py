"""Host-side logic of a multi-process run where every rank advances its own
independent lattice (the method has no exchange step between independent
media, so ranks share nothing but the timing).

``aggregate`` turns per-rank work and per-rank device time into the
whole-job figures: the job time is the slowest rank's, the work is the sum.
"""
from __future__ import annotations

import os


def rank_info() -> tuple[int, int, int]:
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def aggregate(units: float, seconds: float, group=None) -> tuple[float, float]:
    """Sum of units over ranks and max of seconds over ranks.

    With a single process (no initialised process group) it returns its
    arguments.  ``group`` is a torch.distributed group (default: world)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return units, seconds
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(u.item()), float(t.item())


def barrier(group=None) -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier(group=group)
