"""Host-side helpers for runs with one process per GPU (torch.distributed).

The single-tree M2L step has no exchange in this library: every rank runs its
own replica, and a whole-job rate is the work of all ranks divided by the
slowest rank's time.  The batched path shards independent problems across
ranks (problem i goes to rank i mod world), again with no data exchange.  Only
these scalar reductions cross ranks; they run on whatever backend the process
group uses (NCCL between GPUs, gloo on CPU).
"""
from __future__ import annotations


def world():
    """(world size, rank) of the default process group, or (1, 0) without one."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(), dist.get_rank()
    return 1, 0


def shard(n: int, rank: int, world_size: int):
    """Indices of the problems that `rank` runs out of `n` independent problems."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError(f"rank {rank} outside a world of {world_size}")
    return list(range(rank, n, world_size))


def _reduce(x: float, op_name: str) -> float:
    import torch
    import torch.distributed as dist

    ws, _ = world()
    if ws == 1:
        return float(x)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name))
    return float(t.item())


def max_over_ranks(x: float) -> float:
    """The slowest rank's value (timings)."""
    return _reduce(x, "MAX")


def sum_over_ranks(x: float) -> float:
    """The sum over ranks (work done)."""
    return _reduce(x, "SUM")


def job_rate(units_this_rank: float, seconds_this_rank: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return sum_over_ranks(units_this_rank) / max_over_ranks(seconds_this_rank)
