"""Autotuner of the FP32 octree rounds: per network, the noise-column count K
of affine-truncate (Sec. 3.3) and the SIMT tile shape (threads per CTA, so
boxes per CTA = threads / padded width).

K trades cost per box against tightness: more kept symbols cost more per box
but leave fewer boxes UNKNOWN, and every UNKNOWN box spawns eight more at the
next level of Proc. 3. The tuner measures both on the GPU: it builds the
network's own frontier at a probe level, times one classify-and-split round
of that frontier for every feasible (K, threads) pair with CUDA events, and
reads each K's UNKNOWN fraction u_K. It then picks the pair that minimises the
modelled cost of the rest of the tree,

    t(K, threads) * sum_{j=0}^{D - probe} (8 u_K)^j,

the measured time per node times the expected number of descendants each
probe-level node still costs down to depth D (a branching process with the
probe level's UNKNOWN fraction). Ties go to the smaller K.
"""
from __future__ import annotations

import numpy as np
import torch

from . import sra

K_CHOICES = (16, 32, 64, 128)
THREAD_CHOICES = (128, 256, 512, 1024)


def max_threads(K):
    """Threads per CTA the FP32 engine allows for this noise-column bound."""
    return 256 if K >= 64 else (512 if K >= 32 else 1024)


def padded_width(mlp):
    w = max([mlp.widths[0]] + list(mlp.widths[1:-1]))
    return (w + 31) // 32 * 32


def candidates(mlp, ks=K_CHOICES, threads=THREAD_CHOICES):
    """Feasible (K, threads per CTA) pairs: the padded width fits the CTA."""
    H = padded_width(mlp)
    out = []
    for K in ks:
        mt = max_threads(K)
        if H > mt:
            continue
        ts = sorted({t for t in threads if H <= t <= mt} | {H})
        for t in ts:
            out.append((K, t))
    return out


def probe_frontier(net, level, cap, K=16):
    """The network's frontier at `level` (affine-truncate K), at most cap nodes."""
    o = sra.make_opts(arith="truncate", K=K)
    fr = torch.zeros((1, 4), dtype=torch.int16, device="cuda")
    for lv in range(level):
        out, _, cnt = sra.classify_and_split(net, fr, 16, opts=o)
        nc = int(cnt[sra.CNT_CHILDREN].item())
        if nc == 0:
            return fr, lv
        fr = out[:min(nc, cap)].contiguous()
    return fr, level


def time_round(net, fr, opts, reps):
    """Median CUDA-event time (ms) of one classify-and-split round of fr."""
    n = fr.shape[0]
    out = torch.empty((8 * n, 4), dtype=torch.int16, device="cuda")
    counts = torch.zeros(sra.CNT_N, dtype=torch.int64, device="cuda")
    sra.classify_and_split(net, fr, 16, opts=opts, out=out, counts=counts)  # warm-up
    ts = []
    for _ in range(reps):
        counts.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        sra.classify_and_split(net, fr, 16, opts=opts, out=out, counts=counts)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    u = float(counts[sra.CNT_UNKNOWN].item()) / n
    return float(np.median(ts)), u


def tune(net, mlp, depth, probe_level=4, sample=2048, reps=3, ks=K_CHOICES, threads=THREAD_CHOICES):
    """Choose (K, threads per CTA) for building this network's tree to depth.
    Returns {"K", "block_threads", "probe_level", "table": [...]}."""
    fr, lv = probe_frontier(net, probe_level, sample)
    n = fr.shape[0]
    remaining = max(depth - lv, 0)
    table, u_of = [], {}
    for K, t in candidates(mlp, ks, threads):
        ms, u = time_round(net, fr, sra.make_opts(arith="truncate", K=K, block_threads=t), reps)
        u_of[K] = u
        b = 8.0 * u
        expand = sum(b ** j for j in range(remaining + 1))
        table.append({"K": K, "block_threads": t, "ms": ms, "ms_per_node": ms / n, "unknown_frac": u,
                      "model_cost": ms / n * expand})
    best = min(table, key=lambda r: (r["model_cost"], r["K"], r["block_threads"]))
    return {"K": best["K"], "block_threads": best["block_threads"], "probe_level": lv,
            "probe_nodes": n, "table": table}
