"""Weak scaling over ranks: the path has no exchange step.

Independent problems (wavelength points of a batch, or replicas of one
problem) are split across ranks, each rank solves its share on its own
GPU, and the only cross-rank traffic is a barrier and a max over ranks of
the elapsed time (no data-path collective).  Wavelengths are dealt
largest-first round-robin so every rank gets a similar amount of work.
"""

from __future__ import annotations

from typing import List, Sequence, Tuple


def shard(sizes: Sequence[int], world_size: int, rank: int) -> List[int]:
    """Indices of the problems rank `rank` solves: problems sorted by
    decreasing size, dealt round-robin."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("bad rank / world size")
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    return sorted(order[rank::world_size])


def max_over_ranks(value: float, group=None) -> float:
    """Max of a float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return float(value)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sum_over_ranks(value: float, group=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return float(value)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())


def weak_throughput(units_this_rank: float, ms_this_rank: float, group=None) -> Tuple[float, float]:
    """(whole-job units per second, max elapsed ms): all ranks' units over
    the slowest rank's time."""
    ms = max_over_ranks(ms_this_rank, group)
    units = sum_over_ranks(units_this_rank, group)
    return units / (ms / 1e3), ms
