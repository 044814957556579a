"""Multi-rank helpers: one process per GPU, scenarios sharded across ranks.

Scenarios (and feeders) are independent, so the solve path needs no
collective: each rank solves its own shard.  Collectives appear only around
the timed region (a barrier, max of the timings, sum of the counts) and, if a
caller wants every result on one rank, in gather_shards.
"""
from __future__ import annotations


def shard_range(B: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [lo, hi) of a B-scenario batch owned by rank (sizes differ by at most 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    q, r = divmod(B, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def rank_seed(seed: int, rank: int) -> int:
    """Seed of rank's own synthetic scenario batch in weak-scaling runs."""
    return seed + 7919 * rank


def reduce_max(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_shards(local, B: int, device=None):
    """All ranks' shards of a [B, ...] result, concatenated in scenario order on every rank.

    local: this rank's shard (rows shard_range(B, rank, world)).
    """
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return local
    world = dist.get_world_size()
    sizes = [shard_range(B, r, world) for r in range(world)]
    rest = tuple(local.shape[1:])
    m = max(hi - lo for lo, hi in sizes)
    pad = torch.zeros((m,) + rest, dtype=local.dtype, device=device)
    pad[:local.shape[0]] = local
    bufs = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(bufs, pad)
    return torch.cat([bufs[r][:hi - lo] for r, (lo, hi) in enumerate(sizes)], dim=0)
