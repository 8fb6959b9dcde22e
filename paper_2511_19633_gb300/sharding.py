"""Event sharding across ranks (one process per GPU).

Events are independent and every random number is keyed by the event id
(Sec. 2, Sec. 4.3: the paper runs independent event samples per node and
merges histograms afterwards), so N ranks take disjoint contiguous event
ranges and exchange nothing on the data path; only the step time (max over
ranks) and, when wanted, the histograms (sum over ranks) are reduced.
"""
from __future__ import annotations


def rank_first_event(rank: int, step: int, events_per_step: int, steps_total: int, base: int = 0) -> int:
    """First event id of (rank, step): rank r owns ids
    base + [r * steps_total * E, (r + 1) * steps_total * E), step k the k-th
    block of E of them."""
    if rank < 0 or step < 0 or step >= steps_total or events_per_step < 0:
        raise ValueError("bad rank/step")
    return base + (rank * steps_total + step) * events_per_step


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank scalar (the step time) over the process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_histograms(tensors, dist=None):
    """In-place sum of histogram tensors over the process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return tensors
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return tensors
