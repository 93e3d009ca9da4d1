"""Data-parallel replicas across GPUs (one process per GPU).

The frames of a job are independent, so ranks need no data exchange: every
rank detects its own frames, and the only collectives are a barrier around
the timed region and a maximum of the ranks' times.  The job's throughput is
the frames of all ranks over the slowest rank's time (weak scaling).
"""
from __future__ import annotations

import os


def env_rank() -> tuple[int, int, int]:
    """(rank, local rank, world size) from the launcher's environment."""
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def frame_seeds(rank: int, n: int, seed0: int = 1002) -> list[list[int]]:
    """Seeds of rank ``rank``'s n frames: disjoint across ranks."""
    return [[seed0 + 1000 * rank, i] for i in range(n)]


def max_over_ranks(x: float, dist=None, device: str = "cpu") -> float:
    """The maximum of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units of all ranks per second of the slowest rank."""
    return units_per_rank * world / seconds
