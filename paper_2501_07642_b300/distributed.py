"""Draw-range sharding of one accepted pool over several ranks.

Candidate draws are independent, so a pool of B draws splits into contiguous draw
ranges, one per rank (the paper names multi-device candidate generation as future
work, Sec. 5). For the best-K rule every rank keeps its own best K -- with K the
global count, because the global best K may all lie in one shard -- and one exchange
(an all-gather of K x 16 bytes per rank) plus a merge by (M, draw index) gives exactly
the pool a single device would accept. Threshold pools need no merge beyond a union.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["shard", "global_k", "shard_q", "merge_accepted", "select_sharded"]


def shard(B_total: int, rank: int, world: int) -> tuple[int, int]:
    """(offset, count) of rank's contiguous share of [0, B_total)."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    base, extra = divmod(B_total, world)
    off = rank * base + min(rank, extra)
    return off, base + (1 if rank < extra else 0)


def global_k(q: float, B_total: int) -> int:
    """K = ceil(qB - 1e-9 qB), clamped to [1, B] (the acceptance count of a pool)."""
    qb = q * B_total
    return int(min(max(math.ceil(qb - 1e-9 * qb), 1), B_total))


def shard_q(K: int, count: int) -> float:
    """The acceptance probability that makes a shard of `count` draws keep K of them."""
    return min(1.0, K / count)


def merge_accepted(parts, K: int | None):
    """Merge per-shard accepted lists [(keys, M64), ...] into the pool: with K, the K
    smallest (M64, key); without K (threshold pools), the union. Returned sorted by key."""
    keys = np.concatenate([np.asarray(p[0], dtype=np.uint64) for p in parts]) if parts else np.zeros(0, np.uint64)
    m = np.concatenate([np.asarray(p[1], dtype=np.float64) for p in parts]) if parts else np.zeros(0)
    if K is not None:
        order = np.lexsort((keys, m))[:K]
        keys, m = keys[order], m[order]
    order = np.argsort(keys, kind="stable")
    return keys[order], m[order]


def select_sharded(ctx, seed: int, first: int, B_total: int, q: float | None = None, threshold: float | None = None,
                   group=None):
    """frr_select over this rank's share of [first, first + B_total), then the exchange.
    Uses torch.distributed (any backend) when initialised, else runs as one rank."""
    from . import frr
    import torch.distributed as dist

    world = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
    rank = dist.get_rank(group) if world > 1 else 0
    off, count = shard(B_total, rank, world)
    K = None if q is None else global_k(q, B_total)
    if count > 0:
        lq = None if q is None else shard_q(K, count)
        keys, m = frr.frr_select(ctx, seed, first + off, count, q=lq, threshold=threshold)
        part = (np.array(keys), np.array(m))
    else:
        part = (np.zeros(0, np.uint64), np.zeros(0))
    if world == 1:
        return merge_accepted([part], K)
    gathered = [None] * world
    dist.all_gather_object(gathered, part, group=group)
    return merge_accepted(gathered, K)
