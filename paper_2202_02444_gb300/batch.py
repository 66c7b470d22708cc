"""Fixed-depth trees (Proc. 3) of many networks at once: every level of every
network's tree goes through one batched round (sra_classify_and_split_batch),
so a level of all networks costs a handful of launches instead of four per
network. The children of network k land contiguously in the round's output
buffer and are the next round's segment k directly (no gather).

A network whose next frontier would exceed `cap` nodes stops there and is
reported as truncated (the frontier budget of build_trees)."""
from __future__ import annotations

import numpy as np
import torch

from . import sra


def build_trees(nets, opts, depths, cap=500_000, root_lo=(-1.0, -1.0, -1.0), root_hi=(1.0, 1.0, 1.0)):
    """Returns per network: leaves (UNKNOWN nodes at its depth), nodes bounded,
    per-level [pos, neg, unk] counts, truncated flag; plus rounds run."""
    k = len(nets)
    fan = [8 if o.split == 0 else 2 for o in opts]
    frontier = torch.zeros((k, 4), dtype=torch.int16, device="cuda")  # one root per network
    seg_first = list(range(k))
    seg_n = [1] * k
    level = [0] * k
    active = [depths[j] >= 0 for j in range(k)]
    res = [{"leaves": 0, "nodes": 0, "levels": [], "truncated": False} for _ in range(k)]
    rounds = 0
    while any(active):
        segs, idx, out_first, leaf_first = [], [], 0, 0
        for j in range(k):
            if not active[j]:
                continue
            at_depth = level[j] >= depths[j]
            cap_out = 0 if at_depth else fan[j] * seg_n[j]
            segs.append(sra.BatchSeg(net=j, max_level=depths[j], first=seg_first[j], n=seg_n[j],
                                     out_first=out_first, cap_out=cap_out, leaf_first=leaf_first,
                                     cap_leaves=seg_n[j] if at_depth else 0))
            idx.append(j)
            out_first += cap_out
            leaf_first += seg_n[j] if at_depth else 0
        out = torch.empty((max(out_first, 1), 4), dtype=torch.int16, device="cuda")
        leaves = torch.empty((max(leaf_first, 1), 4), dtype=torch.int16, device="cuda")
        counts = sra.classify_and_split_batch(nets, opts, frontier, segs, out, leaves,
                                              root_lo=root_lo, root_hi=root_hi)
        cnt = counts.cpu().numpy()
        rounds += 1
        for s, j in enumerate(idx):
            c = cnt[s]
            r = res[j]
            r["nodes"] += seg_n[j]
            r["levels"].append([int(c[sra.CNT_POSITIVE]), int(c[sra.CNT_NEGATIVE]), int(c[sra.CNT_UNKNOWN])])
            if level[j] >= depths[j]:
                r["leaves"] = int(c[sra.CNT_LEAVES])
                active[j] = False
                continue
            children = int(c[sra.CNT_CHILDREN])
            if children == 0:
                active[j] = False
                continue
            if children > cap:
                r["truncated"] = True
                active[j] = False
                continue
            seg_first[j] = segs[s].out_first
            seg_n[j] = children
            level[j] += 1
        frontier = out
    return res, rounds


def build_trees_one_by_one(nets, opts, depths, cap=500_000):
    """The same trees, one network and one level at a time (lone rounds)."""
    res = []
    for net, o, depth in zip(nets, opts, depths):
        fr = torch.zeros((1, 4), dtype=torch.int16, device="cuda")
        r = {"leaves": 0, "nodes": 0, "levels": [], "truncated": False}
        for lv in range(depth + 1):
            out, lf, cnt = sra.classify_and_split(net, fr, depth, opts=o)
            c = cnt.cpu().numpy()
            r["nodes"] += fr.shape[0]
            r["levels"].append([int(c[sra.CNT_POSITIVE]), int(c[sra.CNT_NEGATIVE]), int(c[sra.CNT_UNKNOWN])])
            if lv == depth:
                r["leaves"] = int(c[sra.CNT_LEAVES])
                break
            ch = int(c[sra.CNT_CHILDREN])
            if ch == 0:
                break
            if ch > cap:
                r["truncated"] = True
                break
            fr = out[:ch]
        res.append(r)
    return res
