"""Several GPUs of one node: one process per GPU. A single system is run as
replicas (each rank its own seeded instance); a batch of independent systems
is dealt out across the ranks.

Instances are independent problems, so ranks exchange nothing on the data
path; the only collectives are the barrier around the timed region and the
maximum of the elapsed times, from which the whole-job throughput is formed.
"""
from __future__ import annotations

import os


def rank_env():
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def instance_of(rank: int) -> int:
    """Seed instance of the workload handled by a rank (distinct per rank)."""
    return rank


def shard(items, rank: int, world: int):
    """The items of one rank when independent problems are dealt round-robin
    (item k to rank k mod world): disjoint, and together all items."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    return list(items)[rank::world]


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (the slowest rank's elapsed time)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Units processed by all ranks per second of the slowest rank."""
    return world * units_per_rank / (ms_max / 1e3)
