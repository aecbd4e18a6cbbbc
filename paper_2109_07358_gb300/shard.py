"""Sharding of a sampling job over ranks.

Samples are independent and each is keyed by (seed, global sample index), so a job of
`total` samples splits into contiguous index ranges, one per rank, with U replicated
and no collective on the data path.  Gathering the results is optional and happens
once at the end (``gather``).
"""
from __future__ import annotations


def shard_range(total: int, rank: int, world: int) -> tuple[int, int]:
    """[lo, hi) of rank `rank` when `total` samples are split over `world` ranks
    (the first total % world ranks take one extra sample)."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, total >= 0")
    base, extra = divmod(total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def step_offset(step: int, rank: int, world: int, per_rank: int) -> int:
    """First global sample index of `rank` at bench step `step` (weak scaling: every
    rank draws `per_rank` new samples per step, ranges never overlap)."""
    return (step * world + rank) * per_rank


def gather(local, total: int, group=None):
    """All-gather the per-rank sample blocks (torch tensors, rows = samples) into the
    full (total, ...) array in global index order."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    sizes = [shard_range(total, r, world) for r in range(world)]
    width = max(hi - lo for lo, hi in sizes)
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[: hi - lo] for p, (lo, hi) in zip(parts, sizes)])
