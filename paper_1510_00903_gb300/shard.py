"""Weak-scaling placement of independent correlator units on ranks.

The correlators of one (gauge configuration, wall source) pair need nothing
from any other pair (Sec. 5 averages over many sources and configurations),
so a multi-GPU job shards those units over the ranks with no exchange on the
data path.  The only collectives are the barrier around the timed region and
the max-over-ranks reduction of its duration.  One process per GPU.
"""
from __future__ import annotations


def units_of_rank(n_units: int, rank: int, world: int) -> list[int]:
    """Round-robin share of units 0..n_units-1 for ``rank`` (disjoint over
    ranks, together every unit exactly once)."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError("need 0 <= rank < world and n_units >= 0")
    return list(range(rank, n_units, world))


def rank_source(rank: int) -> dict:
    """Synthetic-input keys of the wall source a rank computes in the weak-
    scaling workload: its own source index and seed, so every rank's
    propagators are independent draws."""
    return {"seed": 1000 + rank, "source": rank}


def barrier(world: int, timeout_s: float | None = None):
    """All ranks meet.  With ``timeout_s`` (gloo process groups) a rank that
    does not arrive in time -- it failed, exited or hangs between steps --
    makes the call raise RuntimeError naming it, instead of waiting forever:
    the surviving ranks learn of the failure on the host before their next
    launch."""
    if world > 1:
        import torch.distributed as dist
        if timeout_s is None:
            dist.barrier()
        else:
            import datetime
            dist.monitored_barrier(timeout=datetime.timedelta(seconds=timeout_s))


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Maximum of ``x`` over all ranks (the job's time is its slowest rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job units per second: every rank's units over the slowest rank's
    time per step."""
    if ms_max <= 0:
        raise ValueError("step time must be positive")
    return world * units_per_rank / (ms_max / 1e3)
