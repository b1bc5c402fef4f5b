"""Replicas across GPUs of one node.

Frames are independent (each is its own CFAR problem), so N GPUs run N
independent copies of the chain: one process per GPU (torchrun), each on its
own frames, with no collective on the data path. These helpers are the host
side of that: process-group set-up from the torchrun environment, the
partition of a frame list over ranks, a barrier, and the maximum over ranks
of a time (the job's time is its slowest rank's).
"""
from __future__ import annotations

import os


def setup(backend: str | None = None):
    """(rank, world, local_rank, torch.distributed or None) from RANK / WORLD_SIZE /
    LOCAL_RANK / MASTER_ADDR / MASTER_PORT. NCCL when CUDA is available, else gloo."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world <= 1:
        return rank, world, local, None
    import torch
    import torch.distributed as dist
    if backend is None:
        backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    if not dist.is_initialized():
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return rank, world, local, dist


def shard(n_items: int, rank: int, world: int) -> range:
    """Contiguous block of item indices for this rank; block sizes differ by at most one."""
    if world < 1 or not (0 <= rank < world) or n_items < 0:
        raise ValueError("bad rank / world / item count")
    base, extra = divmod(n_items, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def barrier(dist) -> None:
    if dist is not None:
        dist.barrier()


def max_over_ranks(x: float, dist) -> float:
    """Maximum of a host float over all ranks (identity without a process group)."""
    if dist is None:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, dist) -> float:
    """Sum of a host float over all ranks (identity without a process group)."""
    if dist is None:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
