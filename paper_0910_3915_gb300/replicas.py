"""Host logic of the multi-GPU runs: independent replicas, one per rank.

The step has no exchange between ranks when each rank advances its own
lattices (a droplet per rank, or a shard of a sweep's boxes), so ranks share
nothing on the data path. They meet only to time the job: a barrier on both
sides of the timed region, the slowest rank's time, and the units all ranks
processed. Launched by torch.distributed.run (RANK, LOCAL_RANK, WORLD_SIZE,
MASTER_ADDR, MASTER_PORT from the environment).
"""
from __future__ import annotations

import os


def world():
    """(world_size, rank, local_rank) from the launcher's environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(items, rank: int, world_size: int):
    """Round-robin share of `items` for `rank`: every item on exactly one rank."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("rank must lie in [0, world_size)")
    return list(items)[rank::world_size]


def whole_job(units: float, seconds: float, device=None):
    """(total units over all ranks, slowest rank's seconds). Without an
    initialised process group this is the rank's own pair. `device` holds the
    reduction tensors (a CUDA device for NCCL, None for CPU backends)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(units), float(seconds)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


def barrier():
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
