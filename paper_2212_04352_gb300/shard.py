"""Sharding of independent fTWA samples over ranks (host logic only).

Samples are independent trajectories, and sample m is a pure function of
(seed, m) (Philox counters are keyed by the global sample index), so ranks
take disjoint contiguous sample ranges.  The only exchange step is at the
end: each rank's estimators (Eq. 5) over its own samples are combined into
the estimators over the union of all ranks' samples by two all-reduces of
their sufficient statistics (combine_moments); timings are reduced by a max.
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


def combine_moments(M, occ, conn, world, want_g2=True):
    """Estimators over the union of every rank's samples from each rank's own
    estimators over its M samples (Eq. 5: occ = mu + 1/2 and the connected
    correlator conn = mean((x - mu)(x - mu)^T); Eq. 10: g2).

    Exchange step of the sample-parallel path: all-reduce of M and M mu,
    then of M (conn + (mu - mu_all)(mu - mu_all)^T) around the combined mean
    (the pairwise form of the pooled covariance, without the cancellation of
    raw second moments).  Tensors [T, K] and [T, K, K] float64 on the
    backend's device (CUDA for NCCL, CPU for gloo); world == 1 returns the
    inputs' values.  Returns (M_total, occ, conn, g2 or None)."""
    import torch
    mu = occ - 0.5
    m = torch.tensor([float(M)], dtype=torch.float64, device=occ.device)
    s1 = mu * float(M)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(m)
        dist.all_reduce(s1)
    M_all = m.item()
    mu_all = s1 / M_all
    d = mu - mu_all
    s2 = (conn + d[:, :, None] * d[:, None, :]) * float(M)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(s2)
    conn_all = s2 / M_all
    occ_all = mu_all + 0.5
    g2 = None
    if want_g2:
        nn = occ_all[:, :, None] * occ_all[:, None, :]
        g2 = (conn_all + nn) / nn
    return int(round(M_all)), occ_all, conn_all, g2
