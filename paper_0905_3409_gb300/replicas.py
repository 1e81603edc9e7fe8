"""Replica runs on several GPUs of one node (one process per GPU, launched by torchrun).

The GALS step runs one grid per GPU: there is no data-path collective.  A run on N GPUs
advances N independent replicas; the only communication is the timing protocol of the
benchmark: a barrier on both sides of the timed region and the maximum of the per-rank
times, so that the whole-job throughput is (units processed by all ranks) / (slowest
rank's time).  The functions take the process group backend as an argument, so the same
host logic runs on NCCL (GPU) and on gloo (CPU tests).
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass
class Ranks:
    rank: int
    world: int
    local: int
    dist: object = None  # torch.distributed when world > 1, else None

    @property
    def leader(self) -> bool:
        return self.rank == 0


def init(backend: str = "nccl") -> Ranks:
    """Rank, world size and local rank from the torchrun environment; initialises the
    process group (backend `backend`) when there is more than one rank."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return Ranks(rank, world, local, dist)


def barrier(r: Ranks) -> None:
    if r.dist is not None:
        r.dist.barrier()


def max_over_ranks(r: Ranks, value: float, device: str = "cpu") -> float:
    """The maximum of `value` over all ranks (every rank gets it)."""
    if r.dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    r.dist.all_reduce(t, op=r.dist.ReduceOp.MAX)
    return float(t.item())


def throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput of N replicas that each processed `units_per_rank` units in at
    most `seconds` (the slowest rank's time)."""
    return units_per_rank * world / seconds


def finish(r: Ranks) -> None:
    if r.dist is not None and r.dist.is_initialized():
        r.dist.destroy_process_group()
