"""Sharding of independent range-analysis work across processes.

Every box, tree node and ray is bounded independently (Proc. 1-3), so N
processes (one per GPU) split the work into contiguous shards and need no
collective on the data path; only per-shard tallies are combined afterwards.
"""
from __future__ import annotations


def shard_range(n: int, rank: int, world: int):
    """[start, stop) of shard `rank` when n items are split over `world`
    processes as evenly as possible (the first n % world shards get one more)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard arguments")
    q, r = divmod(n, world)
    start = rank * q + min(rank, r)
    stop = start + q + (1 if rank < r else 0)
    return start, stop


def weak_shard(n_per_rank: int, rank: int):
    """[start, stop) of this rank's fixed-size batch in a global batch of
    n_per_rank * world items (weak scaling: work per process is constant)."""
    return rank * n_per_rank, (rank + 1) * n_per_rank
