"""Replica sharding across ranks (one process per GPU).

Trajectories are independent and their random streams are keyed by the
global replica index (cwc_sim_args.replica_offset), so a shard is just a
contiguous replica range; there is no exchange on the data path.  Only the
throughput figures are combined: events are summed and the time is the
slowest rank's.
"""
from __future__ import annotations

from typing import Optional, Tuple


def weak_shard(replicas_per_rank: int, rank: int) -> Tuple[int, int]:
    """(replica_offset, count) of rank's shard when every rank runs the same number of replicas."""
    return rank * replicas_per_rank, replicas_per_rank


def strong_shard(total_replicas: int, world: int, rank: int) -> Tuple[int, int]:
    """(replica_offset, count) of rank's part of a fixed total, as even as possible."""
    base, extra = divmod(total_replicas, world)
    off = rank * base + min(rank, extra)
    return off, base + (1 if rank < extra else 0)


def combine(events: float, seconds: float, group=None, device: Optional[str] = None) -> Tuple[float, float]:
    """Sum of events over ranks and the maximum time (torch.distributed; identity when not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return events, seconds
    ev = torch.tensor([float(events)], dtype=torch.float64, device=device)
    tm = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(ev, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX, group=group)
    return float(ev.item()), float(tm.item())
