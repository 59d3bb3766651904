"""Data-parallel split of one fitting step over ranks (one GPU each).

The render step shards over views (cameras x frames): every rank holds the
whole atlas, renders and back-propagates its own views, and the texel
gradients of all ranks are summed -- the one exchange of the step.  These
helpers hold that host-side logic; the kernels are the same on every rank.
"""

from __future__ import annotations

from typing import List, Sequence


def shard_views(views: Sequence, rank: int, world: int) -> List[int]:
    """Indices of the views rank `rank` of `world` renders.

    Views are dealt greedily by pixel count (largest first, each to the
    least-loaded rank, ties to the lower rank), so the shards cover every
    view exactly once and their pixel totals differ by at most one view.
    The result is ordered by view index and identical on every rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} of world {world}")
    order = sorted(range(len(views)), key=lambda i: (-int(views[i].width) * int(views[i].height), i))
    load = [0] * world
    owner = [0] * len(views)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += int(views[i].width) * int(views[i].height)
    return [i for i in range(len(views)) if owner[i] == rank]


def allreduce_texel_grads(grad, group=None):
    """Sum the texel gradients of every rank in place (the step's exchange)."""
    import torch.distributed as dist
    dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    return grad


def max_over_ranks(value: float, group=None) -> float:
    """The slowest rank's time (what a synchronous step waits for)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
