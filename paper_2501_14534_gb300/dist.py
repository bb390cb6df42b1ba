"""Multi-process helpers (one process per GPU, torch.distributed).

The rasterizer itself runs on one GPU. Data-parallel training over views shards the views of
a step across ranks; the one exchange step is then an all-reduce of the per-Gaussian
gradients (sum) and densification statistics (sum of the gradient-norm accumulators and
visibility counts, max of the radii). The benchmark runs independent replicas and only
reduces its timings (max over ranks).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_views(n_views: int, rank: int, world: int):
    """Indices of the views rank renders: a contiguous, balanced block."""
    base, extra = divmod(n_views, world)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))


def reduce_max(x: float, device="cpu") -> float:
    """Maximum of a scalar over all ranks (e.g. the time of a timed region)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_grads(grads: dict, stats: dict | None = None, views_per_rank=None):
    """Sums the gradient tensors over ranks in place, and the statistics (gradient-norm
    accumulator, visibility count and ray hits of the significance score summed, max radius
    maxed).

    With a loss that is a mean over the views of the whole step, each rank's gradients are
    already weighted by 1/(total views); pass ``views_per_rank`` = (this rank's views, total
    views) when each rank normalised by its own view count instead, to rescale before the sum.
    """
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return grads, stats
    scale = None
    if views_per_rank is not None:
        mine, total = views_per_rank
        scale = float(mine) / float(total)
    for t in grads.values():
        if t is None:
            continue
        if scale is not None:
            t.mul_(scale)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    if stats:
        for k in ("grad_norm_accum", "vis_count", "hit_count"):
            if stats.get(k) is not None:
                dist.all_reduce(stats[k], op=dist.ReduceOp.SUM)
        if stats.get("max_radius") is not None:
            dist.all_reduce(stats["max_radius"], op=dist.ReduceOp.MAX)
    return grads, stats
