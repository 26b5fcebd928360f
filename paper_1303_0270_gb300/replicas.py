"""Multi-GPU runs of independent problems (weak scaling, no data-path
collective): one replica per rank, each with its own seeds, timed between
barriers, the job's time being the slowest rank's.  The only communication is
host-side bookkeeping (barrier, max of the times, sum of the work)."""
from __future__ import annotations

import os

import torch


def world():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base: int, rank: int) -> int:
    """Seeds of rank r's replica: the base seeds shifted by 1000 per rank."""
    return base + 1000 * rank


def _reduce(value: float, op, device) -> float:
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(value: float, device="cpu") -> float:
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.MAX if dist.is_available() else None, device)


def sum_over_ranks(value: float, device="cpu") -> float:
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.SUM if dist.is_available() else None, device)


def job_throughput(units_this_rank: float, seconds_this_rank: float, device="cpu") -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    total = sum_over_ranks(units_this_rank, device)
    slowest = max_over_ranks(seconds_this_rank, device)
    return total / slowest
