"""Replica scaling across GPUs of one node.

Rays and frames are independent, so N GPUs render N streams of frames with no
data exchange (weak scaling).  This module holds the host side of that:

* which camera a rank renders at step j: ranks start at different offsets
  into the camera list and advance by one per step;
* the slowest rank's elapsed time: the only collective, a MAX all-reduce;
* the aggregate rate over all ranks.

It runs on a host (gloo) process group: nothing on the data path crosses GPUs.
"""
from __future__ import annotations


def camera_for(rank: int, step: int, n_cameras: int, stride: int = 7) -> int:
    """Camera index rank `rank` renders at step `step`."""
    return (rank * stride + step) % n_cameras


def max_over_ranks(ms: float, device=None) -> float:
    """The largest `ms` over all ranks (the value itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, max_ms: float, world: int) -> float:
    """Units per second over the whole job: every rank's units over the slowest rank's time."""
    return units_per_rank * world / (max_ms / 1e3)
