"""Multi-GPU execution by replicas.

Chemistry cells are independent (each cell's step reads and writes only its
own state), so N GPUs need no exchange: each rank steps its own cells and
the only collectives are a barrier and the max/sum of timings and counts
around a measurement.  These helpers work with any torch.distributed
backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import os


def rank_env():
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str | None = None):
    world, rank, local = rank_env()
    if world > 1:
        import torch
        import torch.distributed as dist
        if not dist.is_initialized():
            if backend is None:
                backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend)
    return world, rank, local


def shard_range(n: int, rank: int, world: int):
    """Contiguous block of cells [start, stop) of rank out of world (the
    first n % world ranks take one extra cell)."""
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def _reduce(value: float, op, device):
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(value: float, device="cpu") -> float:
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.MAX, device)


def sum_over_ranks(value: float, device="cpu") -> float:
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.SUM, device)


def barrier():
    import torch.distributed as dist
    if dist.is_initialized():
        dist.barrier()
