"""Host logic for running decoder replicas on several GPUs of one node.

Frames are independent, so the decoding path shards by frames with no data-path exchange:
each rank decodes a contiguous share of the frames on its own GPU. The only collectives are
the reductions of per-rank counters (frame errors, frames decoded) and of the per-rank
elapsed time (the job is as slow as its slowest rank).
"""
from __future__ import annotations


def shard(n_total: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous share (start, count) of n_total frames for `rank` of `world`; shares differ
    by at most one frame and cover every frame exactly once."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def allreduce_sum(values, device="cpu"):
    """Element-wise sum over ranks of a list of integers (identity without a process group)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor(list(values), dtype=torch.int64, device=device)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [int(v) for v in t.tolist()]


def allreduce_max(value: float, device="cpu") -> float:
    """Maximum over ranks of a float (the job's elapsed time is its slowest rank's)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
