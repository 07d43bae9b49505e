"""Replica timing across ranks.

Key switching shards across GPUs only by independent operations: every rank
holds its own copy of the keys and runs its own ciphertexts, and no data moves
between ranks. The job's time is therefore the slowest rank's, and its
throughput is all ranks' operations divided by that time (weak scaling: the
work per rank is fixed as ranks are added).
"""
from __future__ import annotations


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def world_size() -> int:
    d = _dist()
    return d.get_world_size() if d else 1


def barrier() -> None:
    """Barrier over the ranks (no-op for one process)."""
    d = _dist()
    if d and d.get_world_size() > 1:
        d.barrier()


def max_over_ranks(value: float) -> float:
    """Maximum of a per-rank scalar over all ranks (the value itself for one
    process). The reduction runs on the GPU for NCCL and on the host for
    gloo."""
    d = _dist()
    if not d or d.get_world_size() == 1:
        return float(value)
    import torch
    dev = "cuda" if d.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    d.all_reduce(t, op=d.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, ms_max: float, world: int) -> float:
    """Units per second of the whole job: every rank processed units_per_rank
    units, and the slowest rank took ms_max milliseconds."""
    if ms_max <= 0:
        raise ValueError("time must be positive")
    return units_per_rank * world / (ms_max / 1e3)
