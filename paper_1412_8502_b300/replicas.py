"""Replica coordination for runs on several GPUs of one node.

The MD path does not shard: independent systems (ensembles, served jobs)
run as replicas, one process per GPU, with no data-path collective.  The
only cross-rank operations are a barrier around the timed region and the
maximum of the ranks' elapsed times, so that whole-job throughput is
(sum of the ranks' units) / (slowest rank's time).  Works with the nccl
backend on GPUs and with gloo on CPU (used by the tests).
"""
from __future__ import annotations

import os


def dist_env():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def init(backend: str = "nccl") -> None:
    import torch.distributed as dist
    _, world, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend)


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(value: float, device: str = "cpu") -> float:
    """Largest value over all ranks (the identity with one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device: str = "cpu") -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units_this_rank: float, ms_this_rank: float, device: str = "cpu") -> float:
    """Units processed by all ranks per second of the slowest rank."""
    units = sum_over_ranks(units_this_rank, device)
    ms = max_over_ranks(ms_this_rank, device)
    return units / (ms * 1e-3)


def replica_seed(seed: int, rank: int) -> int:
    """Distinct, reproducible seed of a rank's replica."""
    return int(seed) + 1000 * int(rank)


def finalize() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()
