"""Host-side logic of the multi-process (one process per GPU) path.

The block transform shards by image: every rank processes its own frames
and there is no data-path collective.  The only cross-rank quantities are
the step time (maximum over ranks, for the throughput of the whole job) and,
when a caller wants one PSNR for the union of all ranks' images, the sum of
(squared error, pixel count).  Both reductions work with any
torch.distributed backend (NCCL on GPUs, gloo in the CPU tests).
"""
from __future__ import annotations

import math


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s synthetic batch (independent batches per rank)."""
    return base + 1000 * rank


def shard(n_items: int, rank: int, world: int):
    """Contiguous share [start, stop) of n_items for a rank (sizes differ by at most one)."""
    q, r = divmod(n_items, world)
    start = rank * q + min(rank, r)
    return start, start + q + (1 if rank < r else 0)


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def max_over_ranks(value: float, device=None) -> float:
    dist = _dist()
    if dist is None or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def global_psnr(sse: float, npix: int, device=None, peak: float = 255.0) -> float:
    """PSNR over the union of all ranks' pixels from per-rank (SSE, pixel count)."""
    dist = _dist()
    s, n = float(sse), float(npix)
    if dist is not None and dist.get_world_size() > 1:
        import torch
        t = torch.tensor([s, n], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        s, n = float(t[0]), float(t[1])
    return math.inf if s == 0.0 else 10.0 * math.log10(peak * peak * n / s)


def job_throughput(units_per_rank_step: float, steps: int, world: int, max_ms: float) -> float:
    """Whole-job rate (units/s x 1e-9) from the slowest rank's time."""
    return units_per_rank_step * steps * world / (max_ms / 1e3) / 1e9
