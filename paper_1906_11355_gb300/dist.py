"""Host-side logic of multi-GPU runs (one process per GPU).

The units of the MCLAHE hot path -- whole volumes -- are independent, so they
are sharded across ranks with no exchange on the data path (weak scaling).
The only collectives are a barrier around the timed region and the
max-over-ranks reduction of the step time; both use whatever process group is
initialised (NCCL on GPUs, gloo on CPUs in the tests).
"""
from __future__ import annotations

import os


def dist_env():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(seed, rank):
    """Seed of a rank's own volume: every rank draws a different volume of
    the same recipe."""
    return int(seed) + 7919 * int(rank)


def shard(sizes, rank, world):
    """Indices of the volumes (given by their sizes) that `rank` processes:
    longest-processing-time-first assignment, so every rank gets about the
    same number of voxels.  Deterministic; every index goes to one rank."""
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    load = [0] * world
    owner = [0] * len(sizes)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += int(sizes[i])
    return [i for i in range(len(sizes)) if owner[i] == rank]


def max_over_ranks(value, device="cpu"):
    """The maximum of a float over all ranks (the value itself without an
    initialised process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms_max):
    """Whole-job throughput in units per second from the slowest rank's time."""
    return float(units_per_rank) * int(world) / (float(ms_max) * 1e-3)
