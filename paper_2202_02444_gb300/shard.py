"""Sharding of independent range-analysis work across processes.

Every box, tree node and ray is bounded independently (Proc. 1-3), so N
processes (one per GPU) split the work into contiguous shards and need no
collective on the data path; only per-shard tallies are combined afterwards.
A frontier is split into contiguous runs of nodes (not round-robin over root
subtrees): a level's frontier is stored in the order of its parents, so a
contiguous run is a set of whole subtrees except at its two ends, and every
node costs the same to bound. Rays are split into contiguous pixel tiles.
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


def rank_batch(frontier, n_per_rank: int, rank: int):
    """This rank's fixed-size batch of a global frontier of n_per_rank * world
    nodes (anything sliceable along its first axis)."""
    a, b = weak_shard(n_per_rank, rank)
    return frontier[a:b]


def rank_ray_tile(width: int, height: int, tile: int, rank: int):
    """Pixel indices (row-major in a width x height image) of this rank's
    tile x tile block of rays: the central block, shifted right by `rank`
    blocks, so that the ranks' tiles are disjoint."""
    x0 = width // 2 - tile // 2 + rank * tile
    y0 = height // 2 - tile // 2
    if x0 < 0 or y0 < 0 or x0 + tile > width or y0 + tile > height:
        raise ValueError("ray tile outside the image")
    return [(y0 + j) * width + (x0 + i) for j in range(tile) for i in range(tile)]
