"""Rank bookkeeping for runs on several GPUs of one node (one process per GPU).

The solver's units of work — independent problems, ensemble members, serving
requests — share nothing, so ranks never exchange state: each rank takes its
own shard of the units, and the only collectives are the barrier around a
timed region and the reductions of its elapsed time and unit counts.  The
functions take the process group that `torch.distributed` was initialised
with (NCCL on GPUs, gloo on CPU); without one they act as a single rank.
"""
from __future__ import annotations

import os


def env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws < 1 or not 0 <= rank < ws or local < 0:
        raise ValueError(f"bad rank environment: WORLD_SIZE={ws} RANK={rank} LOCAL_RANK={local}")
    return ws, rank, local


def shard(n_units: int, rank: int, world: int) -> range:
    """Contiguous share of `n_units` units for `rank` of `world`; shares differ
    by at most one unit, the first `n_units % world` ranks taking the extra."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_units, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def _active():
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def _reduce(value: float, op: str, device) -> float:
    if not _active():
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(value: float, device="cpu") -> float:
    """Largest `value` over all ranks (elapsed times: the job ends with its
    slowest rank)."""
    return _reduce(value, "max", device)


def sum_over_ranks(value: float, device="cpu") -> float:
    """Sum of `value` over all ranks (units processed by the whole job)."""
    return _reduce(value, "sum", device)


def barrier() -> None:
    if _active():
        import torch.distributed as dist
        dist.barrier()


def job_rate(local_units: float, local_seconds: float, device="cpu") -> tuple[float, float]:
    """Whole-job throughput: (units of all ranks) / (slowest rank's time).
    Returns (rate, max seconds)."""
    if local_seconds <= 0:
        raise ValueError("elapsed time must be positive")
    units = sum_over_ranks(local_units, device)
    secs = max_over_ranks(local_seconds, device)
    return units / secs, secs
