"""Multi-GPU runs as independent replicas (the step has no exchange between
lattices): every rank advances its own lattices; ranks only agree on timing and
pool measurements. Collectives here carry measurements, never lattice data."""
from __future__ import annotations


def shard(items, rank, world):
    """The items rank `rank` of `world` takes: every world-th, starting at rank."""
    return list(items)[rank::world]


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Largest value over the ranks (e.g. a timed duration); the value itself when
    not distributed."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_lists(values, dist=None):
    """Concatenation of every rank's list (rank order)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return list(values)
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, list(values))
    return [v for part in out for v in part]
