"""Independent replicas on several GPUs (one process per GPU).

Particles never interact (the paper's Section 3.4: no communication between the
kernels), and the work here is sized for one GPU, so N GPUs run N independent
replicas: rank r simulates its own particles, whose ids start at r * n so that
the counter-based random numbers of different replicas never coincide.  The
only collective is on the timing: the slowest rank's time counts.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def id_offset(rank: int, n_per_rank: int) -> int:
    """First particle id of replica ``rank`` (ids are uint32)."""
    off = int(rank) * int(n_per_rank)
    if off + n_per_rank > 2 ** 32:
        raise ValueError("particle ids of all replicas must fit in 32 bits")
    return off


def max_over_ranks(ms: float) -> float:
    """Largest per-rank time (all ranks call this); identity without a process group."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job rate: units of all replicas over the slowest replica's time."""
    return world * units_per_rank / (ms_max / 1000.0)
