"""Multi-GPU replicas: one process per GPU, each ray-tracing and reducing its
own independent lens system (weak scaling). The data path has no collective;
the only cross-rank operations are the timing barrier and the max-over-ranks
of the step time, which bench.py uses to report whole-job throughput."""
from __future__ import annotations

import os

import torch


def world() -> tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment (1 process if unset)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def rank_seed(rank: int, base: int = 1) -> int:
    """Seed of the lens system a rank owns: distinct per rank, fixed across runs."""
    return base + rank


def max_over_ranks(value: float, device: torch.device | str = "cpu") -> float:
    """Largest value across ranks (the slowest rank's step time); identity with one process."""
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, seconds_max: float, world_size: int) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return world_size * units_per_rank / seconds_max
