"""Multi-GPU use of the library: independent replicas, no collective on the data path.

A single instance does not shard in one exchange step (the K x K Cholesky of
the Schur complement couples every dual variable), so several GPUs are used as
independent replicas: each rank solves its own instances.  The only
communication is host-side bookkeeping after the work: the slowest rank's time
(weak-scaling throughput) and, for families of instances, gathering per-rank
results for reporting.  These helpers work on any torch.distributed backend
(NCCL on GPUs; gloo in the CPU tests).
"""

from __future__ import annotations


def shard(items, rank: int, world: int) -> list:
    """Rank-strided share of a family of independent instances."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return list(items)[rank::world]


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest value over all ranks (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_throughput(units_per_rank: float, local_seconds: float, dist=None, device=None) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    world = dist.get_world_size() if (dist is not None and dist.is_initialized()) else 1
    return world * units_per_rank / max_over_ranks(local_seconds, dist, device)


def gather(obj, dist=None) -> list:
    """Every rank's object, in rank order (reporting only)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out
