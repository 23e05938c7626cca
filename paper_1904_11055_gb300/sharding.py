"""Weak scaling over ranks (one process per GPU).

Each rank takes whole units of work, namely fields or realisations.  No data
moves between ranks: the estimator of one field is independent of every other
field.  The job's time is the slowest rank's.  These helpers are host logic
only.  They work with any torch.distributed backend (NCCL on GPUs, gloo in the
CPU tests), and without an initialised process group they reduce to the
single-rank case.
"""
from __future__ import annotations

import os


def rank_env() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment (torchrun), defaults (0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def unit_range(n_units: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous share [start, stop) of n_units for `rank`; shares differ in size by at most one."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, n_units >= 0")
    return n_units * rank // world, n_units * (rank + 1) // world


def field_seed(base: int, rank: int) -> int:
    """Seed of the field a rank estimates in the weak-scaling run: every rank a distinct field."""
    return base + rank


def _reduce(value: float, op_name: str) -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name))
    return float(t.item())


def max_over_ranks(value: float) -> float:
    """The largest value over all ranks (e.g. the slowest rank's time)."""
    return _reduce(value, "MAX")


def sum_over_ranks(value: float) -> float:
    return _reduce(value, "SUM")


def job_rate(local_units: float, local_seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    total = sum_over_ranks(local_units)
    t = max_over_ranks(local_seconds)
    if t <= 0:
        raise ValueError("the slowest rank's time must be positive")
    return total / t
