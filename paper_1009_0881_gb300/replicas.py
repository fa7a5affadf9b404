"""Multi-GPU layout of independent problems: replicas, no data-path collective.

Each factorisation problem is independent of the others, so several GPUs split a
set of problems between them (one process per GPU) and never exchange factor
data.  The only cross-rank operations are host-side bookkeeping: a barrier
around the timed region and the maximum of the ranks' elapsed times.
"""
from __future__ import annotations


def shard(count: int, rank: int, world: int) -> list[int]:
    """Problem indices owned by `rank`: a contiguous, balanced block of 0..count-1."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(count, world)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))


def replica_seed(rank: int, seed0: int = 1) -> int:
    """Data seed of the problem a rank solves when every rank runs its own copy of the workload."""
    return seed0 + rank


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank float over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(units_per_rank: float, elapsed_ms_per_rank: float, world: int, device=None) -> tuple[float, float]:
    """Whole-job throughput: units all ranks processed over the slowest rank's time.

    Returns (units per second, slowest elapsed ms)."""
    slowest = max_over_ranks(elapsed_ms_per_rank, device)
    return world * units_per_rank / (slowest / 1e3), slowest
