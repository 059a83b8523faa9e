"""Multi-GPU launch logic: one process per GPU, one disorder sample per rank.

The sweep partitions into independent problems (disorder samples and
replicas share nothing), so ranks run with no collective on the data path.
The only collective is the timing reduction: the job's time is the slowest
rank's, and throughput is all ranks' work divided by that time (weak
scaling: fixed work per GPU).
"""
from __future__ import annotations

import os


def env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_sample(rank: int, base_sample: int = 0) -> int:
    """Disorder sample run by `rank`: distinct per rank, so no two ranks
    draw the same couplings or the same Philox stream."""
    return base_sample + rank


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of `value` over all ranks (identity without a process
    group).  `device` is where the reduction tensor lives: a CUDA device for
    NCCL, None (CPU) for gloo."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    if seconds_max <= 0:
        raise ValueError("elapsed time must be positive")
    return units_per_rank * world / seconds_max
