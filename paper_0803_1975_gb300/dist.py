"""Host-side helpers for runs over several GPUs of one node (one process per
GPU, torch.distributed).  The products are independent, so ranks never
exchange data on the compute path: each rank takes a contiguous share of the
units (problems of a batch, or whole replicas of a step) and only the
timings are combined, by a maximum over ranks."""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard(count: int, rank: int, world: int) -> range:
    """Contiguous, balanced share of `count` units for `rank` of `world`
    (shares differ in size by at most one)."""
    if world <= 0 or not (0 <= rank < world) or count < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(count, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks (the value itself without a process
    group)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
