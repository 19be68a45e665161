"""Multi-process (one process per GPU) host logic.

The polynomials of a batch are independent, so ranks never exchange data
inside a step: rank r takes its own index range of the seeded stream (weak
scaling) and builds its own uint32 root-density image. The only exchange is
one element-wise sum of the images (and of the counters) at the end, plus
the maximum of the ranks' timings. The differentiation workload has one more:
its loss compares the soft-density image of all ranks' roots with a target,
so the float64 images are summed (differentiably) before the loss, and each
rank then pulls the gradient back to its own roots.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_range(n_per_rank: int, rank: int):
    """Index range [start, stop) of the seeded stream that `rank` solves."""
    if n_per_rank < 0 or rank < 0:
        raise ValueError("n_per_rank and rank must be >= 0")
    return rank * n_per_rank, (rank + 1) * n_per_rank


def reduce_images(hist: torch.Tensor, dst: int = 0, group=None) -> torch.Tensor:
    """Sum the per-rank histograms into rank `dst` (in place there).

    The images hold uint32 counts in int32 storage; the sum stays exact while
    the total count in any pixel is below 2^31.
    """
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return hist
    dist.reduce(hist, dst=dst, op=dist.ReduceOp.SUM, group=group)
    return hist


def max_over_ranks(value: float, device=None, group=None) -> float:
    """Maximum of a per-rank float (timings: the job is as slow as its slowest rank)."""
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


class _SumOverRanks(torch.autograd.Function):
    """All-reduce (sum) with a gradient: every rank evaluates the same function
    of the summed image, so each already holds the gradient of the global
    loss with respect to the sum, and the sum's adjoint hands it unchanged to
    every rank's own image."""

    @staticmethod
    def forward(ctx, x, group):
        y = x.detach().clone()
        dist.all_reduce(y, op=dist.ReduceOp.SUM, group=group)
        return y

    @staticmethod
    def backward(ctx, grad):
        return grad, None


def global_density(img: torch.Tensor, group=None) -> torch.Tensor:
    """The sum over ranks of the per-rank soft-density images, differentiable
    (one all-reduce forward, none backward). A single process returns img."""
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return img
    return _SumOverRanks.apply(img, group)
