"""Sharding of one RQMC estimate across ranks (one process per GPU).

Every generator on the path is counter-based, so the points i of replication m can be
split into contiguous ranges with no change to any point: a rank prices the range
[offset, offset + count) through the plans' ``offset`` argument, and the estimator of
Sec. 1, theta_N^m = (1/N) sum_i f(q_i^m), is recovered exactly from the per-rank
estimates by the count-weighted mean.  That combination is the only exchange: one
all-reduce of M x n_out doubles.  RQ_{M,N} and its standard error then follow from the
combined theta as on one GPU.
"""
from __future__ import annotations

import torch


def point_range(rank: int, world: int, n_total: int) -> tuple[int, int]:
    """Contiguous share (offset, count) of n_total points for `rank` of `world`; the first
    n_total % world ranks take one extra point."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("need 0 <= rank < world and n_total >= 0")
    base, extra = divmod(n_total, world)
    count = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, count


def combine_theta(theta: torch.Tensor, count: int, group=None, total: int | None = None) -> torch.Tensor:
    """theta_N^m over all ranks' points from this rank's theta (float64, any shape, any
    device the process group supports) over `count` points: sum_r count_r theta_r / sum_r
    count_r.  Every rank returns the combined tensor.  With `total` (= sum_r count_r, known
    on the host when the ranges come from point_range) the combination is one all-reduce of
    theta count / total with no read-back to the host, so several estimates can be combined
    in one call on their concatenation; without it the counts travel with the values."""
    import torch.distributed as dist
    if theta.dtype != torch.float64:
        raise TypeError("theta must be float64")
    if not (dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1):
        return theta.clone()
    if total is not None:
        if total <= 0:
            raise ValueError("no points on any rank")
        w = theta.reshape(-1) * (float(count) / float(total))
        dist.all_reduce(w, op=dist.ReduceOp.SUM, group=group)
        return w.reshape(theta.shape)
    w = torch.cat([theta.reshape(-1) * float(count),
                   torch.tensor([float(count)], dtype=torch.float64, device=theta.device)])
    dist.all_reduce(w, op=dist.ReduceOp.SUM, group=group)
    total_seen = float(w[-1].item())
    if total_seen <= 0:
        raise ValueError("no points on any rank")
    return (w[:-1] / total_seen).reshape(theta.shape)


def rq_stats(theta: torch.Tensor) -> tuple[torch.Tensor, torch.Tensor]:
    """RQ_{M,N} (mean over replications, dim 0) and its standard error (sample std / sqrt M)."""
    M = theta.shape[0]
    rq = theta.mean(dim=0)
    se = theta.std(dim=0, unbiased=True) / M ** 0.5 if M > 1 else torch.zeros_like(rq)
    return rq, se
