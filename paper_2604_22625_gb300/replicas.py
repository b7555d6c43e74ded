"""Replica (weak-scaling) plumbing for multi-GPU runs: one process per GPU,
each solving its own seeded batch, with no collective on the data path.

Only the timing and the solve counts cross ranks: the whole-job value is the
units every rank processed divided by the slowest rank's time.  The helpers
work with any torch.distributed backend (NCCL on GPUs, gloo in the CPU tests).
"""
from __future__ import annotations

import os


def dist_env():
    """(world_size, rank, local_rank) from the torchrun environment."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(base: int, rank: int) -> int:
    """Seed of a rank's batch: rank 0 keeps the workload's own seed."""
    return base + 10 * rank


def _reduce(dist, value: float, device, op):
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(dist, value: float, device="cpu") -> float:
    return _reduce(dist, value, device, dist.ReduceOp.MAX if dist is not None else None)


def sum_over_ranks(dist, value: float, device="cpu") -> float:
    return _reduce(dist, value, device, dist.ReduceOp.SUM if dist is not None else None)


def job_throughput(dist, units: float, seconds: float, device="cpu"):
    """(whole-job units / slowest rank's seconds, slowest seconds, total units)."""
    t = max_over_ranks(dist, seconds, device)
    u = sum_over_ranks(dist, units, device)
    return (u / t if t > 0 else 0.0), t, u
