"""Work split across ranks (one process per GPU).

(frame, view) items are independent given D, so ranks share no data: each rank runs whole frames on its own GPU
and no collective touches the data path.  Frames are dealt to ranks by pixel count (largest first, each to the
least-loaded rank), which keeps uneven resolutions balanced; only the timing is reduced across ranks.
"""
from __future__ import annotations


def assign_frames(pixel_counts: list[int], world: int) -> list[list[int]]:
    """Frame indices per rank; deterministic, every frame exactly once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(pixel_counts)), key=lambda i: (-pixel_counts[i], i))
    load = [0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += pixel_counts[i]
    for lst in out:
        lst.sort()
    return out


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank float (the slowest rank's time); the identity without torch.distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
