"""Multi-GPU runs of the filter are independent replicas (one process per GPU): every rank filters
its own blocks with its own copy of the basis and coefficients, and no collective touches the data
path (blocks are independent units, arXiv:2110.13115 Sec. III.F; the paper batches segments, Sec.
III.E). Only the measurement is combined: the per-step time is the maximum over ranks and the job's
rate counts the units every rank processed."""
from __future__ import annotations


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """Largest `value` over the ranks of the default process group (the value itself alone)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, ms_local: float, dist=None, device="cpu") -> tuple[float, float]:
    """(max over ranks of ms per step, whole-job units per second = world * units / max time)."""
    world = dist.get_world_size() if dist is not None and dist.is_initialized() else 1
    ms = max_over_ranks(ms_local, dist, device)
    return ms, world * units_per_rank / (ms / 1e3)


def rank_share(n_items: int, world: int, rank: int) -> list:
    """Round-robin share of n_items work units (blocks, segments) for `rank` of `world`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world {world}")
    return list(range(rank, n_items, world))
