"""Replica bookkeeping for several GPUs of one node: problems and seeds are
independent with no exchange step, so each rank plans its own problems and only
the timing is combined (the slowest rank sets the whole job's step time)."""
from __future__ import annotations

import torch


def max_over_ranks(value: float, device) -> float:
    """The largest value over the ranks of the default process group (the
    value itself when there is no group)."""
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, ms_per_step_max: float, world: int) -> float:
    """Whole-job rate: the units all ranks processed in one step divided by the
    slowest rank's step time."""
    return units_per_rank * world / (ms_per_step_max * 1e-3)
