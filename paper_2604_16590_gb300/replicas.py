"""Multi-GPU runs of STORM-GPA are replicas: the operator partitions into
independent (batch, head) units with no exchange between them, so each rank
processes its own batch on its own GPU and only the measurement is combined
(no collective on the data path).  These helpers hold that host logic: the
per-rank input seed, and the max-over-ranks / sum-over-ranks reductions of
the timing and the work done (weak scaling: per-GPU work fixed as ranks grow).
"""
from __future__ import annotations

import torch


def replica_seed(base: int, rank: int) -> int:
    """Seed of a rank's inputs (rank 0 uses the workload's own seed)."""
    return int(base) + 1000 * int(rank)


def _reduce(x: float, op, device=None) -> float:
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x: float, device=None) -> float:
    import torch.distributed as dist

    return _reduce(x, dist.ReduceOp.MAX, device)


def sum_over_ranks(x: float, device=None) -> float:
    import torch.distributed as dist

    return _reduce(x, dist.ReduceOp.SUM, device)


def weak_scaling_value(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / max_seconds
