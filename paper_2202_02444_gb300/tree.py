"""Level-synchronous BuildSpatialTree (Proc. 3) with checkpoint and resume.

build_tree runs the tree one level at a time through sra_classify_and_split.
Because the tree is level-synchronous, everything needed to continue after
level k is the frontier of level k + 1, the leaves found so far and the
class counts. With `checkpoint` set, that state is written after every level
(to a temporary file that is then renamed over the checkpoint, so a crash
mid-write leaves the previous checkpoint intact). A later call with the same
checkpoint path continues from the last completed level instead of the root.
The checkpoint records the problem it belongs to: the network's parameters
(a SHA-1 of them), the depth, the root box and the options that change the
tree. Resuming with a different problem is refused.

Each level runs inside an NVTX range ("tree_level_<k>") for profilers, and
with `log` set one JSON line per level is appended to that file: the level,
its frontier size, the POSITIVE / NEGATIVE / UNKNOWN counts, the leaves and
children it produced, the FP64 re-checks and the round's host time.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import numpy as np
import torch

from . import sra

_OPT_FIELDS = ("arith", "K", "slope", "precision", "recheck", "recheck_band", "split", "converge")


def problem_key(mlp, depth, opts, root_lo, root_hi):
    """A string identifying one tree build (the network, depth, root and options)."""
    h = hashlib.sha1()
    h.update(np.ascontiguousarray(mlp.widths, np.int64).tobytes())
    h.update(np.ascontiguousarray(mlp.acts, np.int64).tobytes())
    h.update(np.ascontiguousarray(mlp.params, np.float32).tobytes())
    h.update(str(int(mlp.pe_octaves)).encode())
    fields = ",".join(f"{f}={getattr(opts, f)!r}" for f in _OPT_FIELDS)
    root = ",".join(f"{float(v)!r}" for v in tuple(root_lo) + tuple(root_hi))
    return f"{h.hexdigest()}|depth={int(depth)}|root={root}|{fields}"


def save_state(path, key, level, frontier, leaves, counts):
    """Write one level's state: the next level (level), its frontier and the
    leaves and counts so far (NODE_DTYPE records, int64 counts)."""
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "wb") as f:
        np.savez(f, key=np.array(key), level=np.int64(level), frontier=np.asarray(frontier, sra.NODE_DTYPE),
                 leaves=np.asarray(leaves, sra.NODE_DTYPE), counts=np.asarray(counts, np.int64))
    os.replace(tmp, path)


def load_state(path, key):
    """The state of a checkpoint written for `key`; ValueError for another problem."""
    with np.load(path, allow_pickle=False) as z:
        if str(z["key"]) != key:
            raise ValueError(f"checkpoint {path} belongs to another tree build")
        return (int(z["level"]), z["frontier"].astype(sra.NODE_DTYPE), z["leaves"].astype(sra.NODE_DTYPE),
                z["counts"].astype(np.int64))


def build_tree(net, depth, opts=None, root_lo=(-1.0, -1.0, -1.0), root_hi=(1.0, 1.0, 1.0), checkpoint=None,
               cap=1 << 22, on_level=None, log=None, **kw):
    """Proc. 3 to a fixed depth, one sra_classify_and_split round per level.

    Returns (leaves, counts): the UNKNOWN leaves (NODE_DTYPE records, in the
    order the rounds emit them) and int64 counts of length sra.CNT_N summed
    over the levels (children, leaves, POSITIVE, NEGATIVE, UNKNOWN, re-checked,
    converged). `cap` bounds one level's frontier; a larger one raises SraError
    (SRA_ECAPACITY). on_level(level, n_frontier) is called after each level's
    state is saved."""
    opts = opts or sra.make_opts(**kw)
    key = problem_key(net.mlp, depth, opts, root_lo, root_hi)
    if checkpoint and os.path.exists(checkpoint):
        level, frontier, leaves, counts = load_state(checkpoint, key)
    else:
        level = 0
        frontier = np.zeros(1, sra.NODE_DTYPE)  # the root cell
        leaves = np.zeros(0, sra.NODE_DTYPE)
        counts = np.zeros(sra.CNT_N, np.int64)
    fan = 8 if opts.split == 0 else 2
    dev = torch.device("cuda", torch.cuda.current_device())
    while level <= depth and len(frontier):
        if len(frontier) * fan > cap and level < depth:
            raise sra.SraError(sra.ECAPACITY, f"level {level + 1} frontier would exceed {cap} nodes")
        t0 = time.perf_counter()
        torch.cuda.nvtx.range_push(f"tree_level_{level}")
        fr = sra.nodes_to_tensor(frontier, dev)
        out, lv, cnt = sra.classify_and_split(net, fr, depth, root_lo, root_hi, opts=opts)
        c = cnt.cpu().numpy()
        torch.cuda.nvtx.range_pop()
        if log:
            rec = {"level": level, "frontier": int(len(frontier)), "positive": int(c[sra.CNT_POSITIVE]),
                   "negative": int(c[sra.CNT_NEGATIVE]), "unknown": int(c[sra.CNT_UNKNOWN]),
                   "leaves": int(c[sra.CNT_LEAVES]), "children": int(c[sra.CNT_CHILDREN]),
                   "rechecked": int(c[sra.CNT_RECHECKED]), "converged": int(c[sra.CNT_CONVERGED]),
                   "ms": (time.perf_counter() - t0) * 1e3}
            with open(log, "a") as f:
                f.write(json.dumps(rec) + "\n")
        n_children, n_leaves = int(c[sra.CNT_CHILDREN]), int(c[sra.CNT_LEAVES])
        frontier = sra.tensor_to_nodes(out[:n_children]) if n_children else np.zeros(0, sra.NODE_DTYPE)
        if n_leaves:
            leaves = np.concatenate([leaves, sra.tensor_to_nodes(lv[:n_leaves])])
        counts = counts + c.astype(np.int64)
        level += 1
        if checkpoint:
            save_state(checkpoint, key, level, frontier, leaves, counts)
        if on_level:
            on_level(level, len(frontier))
    return leaves, counts
