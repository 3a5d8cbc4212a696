"""Event-range sharding over ranks (one process per GPU).

Events are independent (Sec. 3 of arXiv:2507.21039: the same branch-free
calculation for every phase-space point), so a batch shards into contiguous
event ranges with no data-path collective; the only exchange is an optional
reduction of two numbers (sum of w |M|^2 and of (w |M|^2)^2) for a
cross-section estimate, or a gather of the per-rank |M|^2 slices.
"""
from __future__ import annotations


def event_range(rank: int, world: int, nevt: int, ev0: int = 0):
    """[lo, hi) of the contiguous block of `nevt` events owned by `rank`;
    the blocks of all ranks tile [ev0, ev0 + nevt) exactly once."""
    if world < 1 or not 0 <= rank < world or nevt < 0:
        raise ValueError("bad shard arguments")
    base, rem = divmod(nevt, world)
    lo = ev0 + rank * base + min(rank, rem)
    hi = lo + base + (1 if rank < rem else 0)
    return lo, hi


def reduce_estimate(weighted_sum: float, weighted_sq: float, count: int):
    """Sum (sum w|M|^2, sum (w|M|^2)^2, events) over ranks (torch.distributed)
    and return the Monte-Carlo mean and its standard error."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([weighted_sum, weighted_sq, float(count)], dtype=torch.float64)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        if dist.get_backend() == "nccl":
            t = t.cuda()
        dist.all_reduce(t)
        t = t.cpu()
    s, s2, n = t.tolist()
    mean = s / n
    var = max(s2 / n - mean * mean, 0.0)
    return mean, (var / n) ** 0.5
