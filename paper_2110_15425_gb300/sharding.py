"""Multi-process layout of the hot path (one process per GPU).

Trials and grid candidates are independent (Sec. 3.6), so the work shards by
contiguous ranges with no exchange for runs; only the grid search's argmax
needs one exchange: each rank's (best value, best index, runner-up) is
gathered and combined with the same lowest-index tie rule as on the device.
"""
from __future__ import annotations


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [lo, hi) of n units for `rank` of `world`; sizes differ by <= 1."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def combine_top2(parts):
    """parts: iterable of (best_value, best_index, second_value); indices are
    global. Returns the merged (best_value, best_index, gap)."""
    best_v, best_i, second = float("-inf"), None, float("-inf")
    for v, i, s in parts:
        if best_i is None:
            best_v, best_i, second = v, i, s
            continue
        if v > best_v or (v == best_v and i < best_i):
            second = max(second, best_v, s)
            best_v, best_i = v, i
        else:
            second = max(second, v)
    gap = 0.0 if second == float("-inf") else best_v - second
    return best_v, best_i, gap


def gather_top2(local, group=None):
    """All-gather each rank's (best_value, best_index, second_value) and merge."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    t = torch.tensor([local[0], float(local[1]), local[2]], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    out = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(out, t, group=group)
    parts = [(float(o[0]), int(o[1]), float(o[2])) for o in out]
    return combine_top2(parts)
