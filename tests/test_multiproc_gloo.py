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

from paper_2202_02444_gb300.shard import shard_range, weak_shard


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
        nodes = wl.random_nodes(n, level=4, seed=12)
        a, b = shard_range(n, rank, world)
        cls, lo, hi, _ = oracle.classify_nodes(wl.net_small_relu(), nodes[a:b], (-1, -1, -1), (1, 1, 1),
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
    cls, *_ = oracle.classify_nodes(wl.net_small_relu(), wl.random_nodes(n, level=4, seed=12),
                                    (-1, -1, -1), (1, 1, 1))
    assert tally == [int((cls == k).sum()) for k in (0, 1, 2)]
    assert sum(sizes) == n and tmax == 2.0
