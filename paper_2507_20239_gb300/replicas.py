"""Replicas across GPUs.

One view's hot path has no exchange step (every stage reads and writes only that
view's records, lists and pixels), so N ranks each render their own view of their
own copy of the scene, with no collective on the data path. The job's rate is the
views of all ranks over the slowest rank's time; these helpers hold that host-side
arithmetic (torch.distributed, any backend) so it can be tested without a GPU.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def world() -> int:
    """Ranks in the default process group (1 without one)."""
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size()
    return 1


def slowest(ms: float, device=None) -> float:
    """The largest of every rank's time (a MAX all-reduce of one number); ms itself
    with a single rank. device: where the reduced tensor lives (the rank's GPU
    under NCCL, the CPU under gloo)."""
    if world() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(views_per_rank: int, n_ranks: int, slowest_ms: float) -> float:
    """Views per second of the whole job: every rank's views over the slowest time."""
    if slowest_ms <= 0:
        raise ValueError("time must be positive")
    return views_per_rank * n_ranks * 1000.0 / slowest_ms
