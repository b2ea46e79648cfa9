"""Replica plan of the multi-GPU mode.

The correlator's streams are independent (no exchange between the F and X
steps is needed when each GPU owns whole streams), so N GPUs run N replicas:
rank r correlates its own stream (seeded per rank), nothing crosses ranks on
the data path, and the job's throughput is all ranks' bytes over the slowest
rank's time.  ``torch.distributed`` is used only for the barrier and for the
max-over-ranks of the timing.
"""

from __future__ import annotations


def rank_seed(base: int, rank: int, stride: int = 100) -> int:
    """Seed of rank ``rank``'s synthetic stream (distinct per rank)."""
    return int(base) + int(stride) * int(rank)


def max_over_ranks(ms: float, dist=None, device=None) -> float:
    """The slowest rank's time (identity on one process)."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(bytes_per_rank: int, world: int, ms: float) -> float:
    """Whole-job GB/s: every rank's bytes over the slowest rank's time."""
    return world * float(bytes_per_rank) / (ms * 1e-3) / 1e9
