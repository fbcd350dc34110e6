"""Sharding of independent fTWA samples over ranks (host logic only).

Samples are independent trajectories, and sample m is a pure function of
(seed, m) (Philox counters are keyed by the global sample index), so ranks
take disjoint contiguous sample ranges and no data-path collective is needed;
only the timing is reduced (max over ranks).
"""

from __future__ import annotations


def sample_range(rank: int, world: int, per_rank: int):
    """(first, count) of the samples owned by `rank` when every rank takes
    `per_rank` samples (weak scaling)."""
    if not (0 <= rank < world) or per_rank < 0:
        raise ValueError("bad rank/world/per_rank")
    return rank * per_rank, per_rank


def split_range(rank: int, world: int, total: int):
    """(first, count) of an even split of `total` samples (strong scaling):
    the first total % world ranks take one extra sample."""
    if not (0 <= rank < world) or total < 0:
        raise ValueError("bad rank/world/total")
    base, extra = divmod(total, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def max_over_ranks(x: float, world: int) -> float:
    """Maximum of a host scalar over the process group (identity for one rank)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
