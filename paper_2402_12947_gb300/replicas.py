"""Replicas-only multi-GPU mode: one process per GPU, each solving its own independent
problem (weak scaling, no data-path collective). This module holds the host-side logic of
that mode: per-rank seeds, the barrier that brackets a timed region, the max-over-ranks
reduction of timings, and the whole-job throughput. It works with any torch.distributed
backend (NCCL on GPUs, gloo on CPU for tests)."""
from __future__ import annotations

import os


def dist_env():
    """(rank, world size, local rank) from the launcher's environment (1 process: 0, 1, 0)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def mesh_seed(base: int, rank: int) -> int:
    """Seed of a rank's meshes: every rank solves a different problem of the same family."""
    return base + 1000 * rank


def rhs_seed(base: int, rank: int) -> int:
    return base + rank


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1 else None


def barrier(cuda: bool = True):
    """Synchronise the device, then every rank (a no-op across ranks for one process)."""
    import torch
    if cuda and torch.cuda.is_available():
        torch.cuda.synchronize()
    dist = _dist()
    if dist is not None:
        dist.barrier()
        if cuda and torch.cuda.is_available():
            torch.cuda.synchronize()


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of floats over all ranks (timings: the job ends when its
    slowest rank ends)."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist = _dist()
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def job_throughput(units_per_rank: float, world: int, ms: float) -> float:
    """Units processed by all ranks per second, with ms the max-over-ranks time of one step."""
    return units_per_rank * world / (ms * 1e-3)
