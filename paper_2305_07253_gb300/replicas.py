"""Running the query on several GPUs of one node: replicas, no data exchange.

Queries are independent (Eq. 1), so each rank traces its own batch against its
own copy of the scene and grid; nothing on the data path is communicated.  The
only collectives are for timing and reporting: a barrier around the timed
region and the maximum of the per-rank times.
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def env() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the torchrun environment (1 process if unset)."""
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def init(backend: str | None = None) -> bool:
    """Join the process group when launched with more than one rank; returns whether it did."""
    _, world, _ = env()
    if world <= 1 or dist.is_initialized():
        return dist.is_initialized()
    dist.init_process_group(backend or ("nccl" if torch.cuda.is_available() else "gloo"))
    return True


def barrier() -> None:
    if dist.is_initialized():
        dist.barrier()
    if torch.cuda.is_available() and torch.cuda.is_initialized():
        torch.cuda.synchronize()


def max_over_ranks(x: float, device: torch.device | None = None) -> float:
    """Largest value of x over all ranks (x itself with one rank)."""
    if not dist.is_initialized():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device: torch.device | None = None) -> float:
    if not dist.is_initialized():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [begin, end) share of n queries for `rank` (sizes differ by at most 1)."""
    base, extra = divmod(n, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def finalize() -> None:
    if dist.is_initialized():
        dist.barrier()
        dist.destroy_process_group()
