"""Two-process (gloo, CPU) checks of the multi-process path: the shards of a
batch partition it, and per-shard tallies merged with all_reduce equal the
tallies of the whole batch (here computed by the FP64 oracle, no GPU)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2202_02444_gb300.shard import rank_batch, rank_ray_tile, shard_range, weak_shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2202_02444_gb300 import workloads as wl
        # the benchmark's split: the frontier is tiled to n_per_rank * world
        # nodes and every rank bounds its own fixed-size batch (rank_batch)
        nodes = wl.random_nodes(n, level=4, seed=12)
        n_per_rank = (n + world - 1) // world
        tiled = np.concatenate([nodes] * 2)[:n_per_rank * world]
        mine = rank_batch(tiled, n_per_rank, rank)
        a, b = weak_shard(n_per_rank, rank)
        cls, lo, hi, _ = oracle.classify_nodes(wl.net_small_relu(), mine, (-1, -1, -1), (1, 1, 1),
                                               nthreads=1)
        tally = torch.tensor([(cls == k).sum() for k in (0, 1, 2)], dtype=torch.int64)
        dist.all_reduce(tally, op=dist.ReduceOp.SUM)
        idx = torch.arange(a, b, dtype=torch.int64)
        sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(sizes, torch.tensor([b - a]))
        t = torch.tensor([float(rank + 1)])
        dist.all_reduce(t, op=dist.ReduceOp.MAX)  # the benchmark's max-over-ranks time
        if rank == 0:
            q.put((tally.tolist(), [int(s) for s in sizes], float(t)))
    finally:
        dist.destroy_process_group()


def test_shard_range_partitions():
    for n in (0, 1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            spans = [shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            for (a0, b0), (a1, b1) in zip(spans, spans[1:]):
                assert b0 == a1
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    assert weak_shard(100, 3) == (300, 400)
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def test_two_process_tallies_merge():
    world, n = 2, 301
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    tally, sizes, tmax = q.get(timeout=10)
    import oracle
    from paper_2202_02444_gb300 import workloads as wl
    n_per_rank = (n + world - 1) // world
    tiled = np.concatenate([wl.random_nodes(n, level=4, seed=12)] * 2)[:n_per_rank * world]
    cls, *_ = oracle.classify_nodes(wl.net_small_relu(), tiled, (-1, -1, -1), (1, 1, 1))
    assert tally == [int((cls == k).sum()) for k in (0, 1, 2)]
    assert sum(sizes) == n_per_rank * world and tmax == 2.0


def test_rank_ray_tiles_are_disjoint():
    tiles = [set(rank_ray_tile(1920, 1080, 64, r)) for r in range(8)]
    assert all(len(t) == 64 * 64 for t in tiles)
    assert len(set().union(*tiles)) == 8 * 64 * 64
    with pytest.raises(ValueError):
        rank_ray_tile(1920, 1080, 64, 20)
