"""Draw-range sharding and the merge exchange (CPU; world size 2 over gloo)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2501_07642_b300.distributed import global_k, merge_accepted, shard, shard_q


def test_shards_cover_the_range_once():
    for B in (1, 7, 100, 200_001):
        for world in (1, 2, 3, 8):
            parts = [shard(B, r, world) for r in range(world)]
            assert sum(c for _, c in parts) == B
            assert all(parts[r][0] + parts[r][1] == parts[r + 1][0] for r in range(world - 1))


def test_shard_q_keeps_global_k():
    for K, count in [(1000, 50_000), (1200, 33_333_334), (2000, 100_000), (5, 3)]:
        qb = shard_q(K, count) * count
        assert min(max(int(np.ceil(qb - 1e-9 * qb)), 1), count) == min(K, count)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, X, n1, seed, B, q, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    Zc, *_ = O.prep(X, "chol")
    K = global_k(q, B)
    off, count = shard(B, rank, world)
    keys, m = O.select(Zc, n1, seed, off, count, q=shard_q(K, count), threads=1)
    gathered = [None] * world
    dist.all_gather_object(gathered, (keys, m))
    if rank == 0:
        out.put(merge_accepted(gathered, K))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_merge_equals_single_pool(oracle):
    X = np.random.default_rng(3).standard_normal((40, 6))
    n1, seed, B, q = 20, 9, 6000, 0.01
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, X, n1, seed, B, q, out)) for r in range(2)]
    for p in procs:
        p.start()
    keys, m = out.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    Zc, *_ = oracle.prep(X, "chol")
    wk, wm = oracle.select(Zc, n1, seed, 0, B, q=q)
    assert np.array_equal(keys, wk) and np.array_equal(m, wm)


def test_merge_threshold_union_and_ties():
    a = (np.array([5, 9], dtype=np.uint64), np.array([1.0, 2.0]))
    b = (np.array([3, 7], dtype=np.uint64), np.array([2.0, 0.5]))
    k, m = merge_accepted([a, b], 3)   # (0.5,7) (1.0,5) (2.0,3) -- the tie at 2.0 goes to key 3
    assert k.tolist() == [3, 5, 7] and m.tolist() == [2.0, 1.0, 0.5]
    k, m = merge_accepted([a, b], None)
    assert k.tolist() == [3, 5, 7, 9]
