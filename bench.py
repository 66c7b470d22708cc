"""Benchmark of the range-analysis hot path on GB300.

One step = one batched octree round of the 3-[256]x8-1 ReLU network
(affine-truncate K=64, FP32, FP64 re-check of near-zero boxes): bound every
node of a frontier batch, classify, compact and split (sra_classify_and_split);
plus one tile of camera rays against the 39(PE)-[512]x6-1 ELU network
(affine-fixed, delta 1e-4; sra_cast_rays). `value` is box-bound evals/s of the
octree part; rays/s is reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2202_02444_gb300 import workloads as wl  # noqa: E402
from paper_2202_02444_gb300.shard import rank_batch, rank_ray_tile  # noqa: E402

BOX_FLOP = None  # filled per net (algorithmic FLOP per box-bound eval)


def box_flops(mlp, K):
    """sum over linear layers of 2 * h_out * h_in * (symbols + 2): the symbol
    columns plus the center and x_inf columns (one box-bound eval)."""
    f = 0
    sym = 3
    for l in range(mlp.n_layers):
        hin, hout = mlp.widths[l], mlp.widths[l + 1]
        f += 2 * hout * hin * (sym + 2)
        sym = K
    return f


def full_flops(mlp):
    """Affine-full: sum over linear layers of 2 * h_out * h_in * (symbols + 1),
    the symbol count growing by h_out after every nonlinear layer."""
    f, sym = 0, 3 + 6 * mlp.pe_octaves
    for l in range(mlp.n_layers):
        hin, hout = mlp.widths[l], mlp.widths[l + 1]
        f += 2 * hout * hin * (sym + 1)
        if l + 1 < mlp.n_layers:
            sym += hout
    return f


def ray_iter_flops(mlp):
    """One CastRay iteration: segment bound (1 symbol + center + x_inf) plus
    the plain point evaluation, through every linear layer."""
    f = 0
    for l in range(mlp.n_layers):
        f += 2 * mlp.widths[l + 1] * mlp.widths[l] * 4
    return f


# DRAM traffic of the dominant kernel's launch in the timed step, from one
# ncu capture of this benchmark (dram__bytes_read.sum + dram__bytes_write.sum,
# 1 pass, NVTX range timed_steps): reported only while the kernel's sources
# are the ones captured (their SHA-1), else null.
TRAFFIC = {
    "tc_bound_kernel<256,true,ReLU>": {"sha1": "e26c3f47f915e507ec9f4b60ba07049751ddb429", "bytes": 2964992,
                                       "capture": "profiles/tc_bound_kernel_bf16_sound_relu256x8_truncate64.md"},
}
TC_BOUND_SOURCES = ("paper_2202_02444_gb300/csrc/tc_bound.cu", "paper_2202_02444_gb300/csrc/tc_bound_impl.cuh",
                    "paper_2202_02444_gb300/csrc/sound_rules.cuh", "paper_2202_02444_gb300/csrc/tc_ptx.cuh",
                    "paper_2202_02444_gb300/csrc/tc_bound.h")


def sources_sha1(paths):
    import hashlib
    h = hashlib.sha1()
    for rel in paths:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def captured_traffic(kernel):
    rec = TRAFFIC.get(kernel)
    if not rec or rec["bytes"] is None or rec["sha1"] != sources_sha1(TC_BOUND_SOURCES):
        return None
    return rec["bytes"]


def measured_peak(key, fallback):
    """A peak from MEASURED_PEAKS.json (copy bandwidth and cuBLAS BF16 measured on this GPU
    model), else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)[key]), "tensor"
    except (OSError, KeyError, ValueError):
        return fallback, "tensor"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--batch", type=int, default=1 << 17, help="octree nodes per step")
    ap.add_argument("--frontier-level", type=int, default=7)
    ap.add_argument("--ray-tile", type=int, default=64, help="ray tile side (tile^2 rays)")
    ap.add_argument("--ray-iters", type=int, default=500, help="per-ray iteration cap of the ray phase")
    ap.add_argument("--ray-complete-cap", type=int, default=40000,
                    help="iteration cap of the ray completion sample (0: skip it)")
    ap.add_argument("--precision", default="bf16_sound", choices=["fp32", "bf16", "bf16_sound"])
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--kernel-case", default=None,
                    choices=["fp32", "bf16_sound", "bf16", "fp64", "rays", "rays_bf16", "full_fp32", "bf16_sound_512",
                             "bf16_sound_k16"],
                    help="run only the bound kernel on --batch boxes of the 256x8 net twice (profiling)")
    ap.add_argument("--serve-rates", default="2,4,8,16", help="request rates (req/s) of the serving sweep")
    ap.add_argument("--serve-requests", type=int, default=32, help="requests per serving trace")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-octree", action="store_true", help="skip the depth-10 octree builds")
    ap.add_argument("--batched-cap", type=int, default=500_000, help="frontier cap per net per level (the batched workload: frontiers of 1k-500k boxes per level)")
    ap.add_argument("--cpu-sample", type=int, default=16384, help="oracle boxes for cpu_baseline")
    ap.add_argument("--cpu-sample-1core", type=int, default=1024,
                    help="oracle boxes for the one-core cpu_baseline figure (0: skip)")
    ap.add_argument("--ref-sample", type=int, default=256, help="oracle boxes per reference step")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu, enabled=True):
        self.gpu, self.enabled, self.proc, self.path = gpu, enabled, None, None

    def __enter__(self):
        if self.enabled:
            self.path = os.path.join("/tmp", f"sra_clocks_{os.getpid()}.csv")
            try:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                     "-lms", "25"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            except OSError:
                self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.remove(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def tc_box_net(m):
    """The network has the tensor-core bound kernel: 3 inputs (no positional
    encoding), 2 to 13 hidden layers of widths up to 512 (run at the width
    128, 256 or 512 that holds them, narrower layers padded with zeros), all
    ReLU, all ELU or all sin, scalar output."""
    return (m.pe_octaves == 0 and m.n_layers >= 3 and m.n_layers - 2 <= 12 and len(set(m.acts)) == 1
            and m.acts[0] in (1, 2, 3) and max(m.widths[1:-1]) <= 512)


def serving_nets():
    """16 resident networks: twelve of the uneven multi-network generator and
    four 39(PE)-[512]x6-1 ELU networks (seeds 2..5)."""
    return [wl.net_batch_mix(i) for i in range(12)] + \
        [wl.make_mlp([512] * 6, "elu", seed=2 + k, pe_octaves=6, name=f"elu_pe6_512x6_s{2 + k}")
         for k in range(4)]


# Resident networks (indices into serving_nets()) whose depth-9 leaf set, in
# affine-truncate K=16 FP32, fits the 2^20-node leaf buffer of a leaf job:
# 65k-900k leaves each. The sin networks of the uneven generator and the
# positional-encoding ELU networks leave nearly every cell UNKNOWN (more than
# 2^20 leaves by depth 7), so a leaf job on them can only end in SRA_ECAPACITY.
SERVING_LEAF_NETS = (3, 4, 6, 8, 9, 11)


def serving_phase(sra, torch, dev, rates, n_req, slots=4, budget=256 << 20):
    """Poisson request traces (seed 5) against 16 resident networks through
    sra_serve: a third each of 64x64 ray tiles (cap 200 iterations per ray),
    batches of U[256, 65536] boxes and leaf-extraction jobs to depth 9 (leaf
    and per-level frontier buffers of 2^20 nodes; the job walks levels that
    are wider in chunks) on the networks of SERVING_LEAF_NETS. Each ray or
    box request takes the BF16-sound form (tensor cores) with probability
    1/2 where its network has that kernel, else FP32.
    Returns p50 / p99 latency (arrival to completion) and throughput per rate."""
    mlps = serving_nets()
    nets = [sra.Net(m) for m in mlps]
    forms = [sra.make_opts(arith="fixed", delta=1e-3, max_iters=200),                     # rays FP32
             sra.make_opts(arith="truncate", K=16),                                       # boxes / leaves FP32
             sra.make_opts(arith="fixed", delta=1e-3, max_iters=200, precision="bf16_sound"),  # rays BF16-sound
             sra.make_opts(arith="truncate", K=64, precision="bf16_sound", recheck=True)]  # boxes BF16-sound

    # the tensor-core ray kernel: hidden widths up to 512 (narrower layers
    # padded with zeros), 1 to 8 hidden-to-hidden layers, at most 64 inputs
    ray_tc = [max(m.widths[1:-1]) <= 512 and 1 <= m.n_layers - 2 <= 8 and m.widths[0] <= 64 for m in mlps]
    box_tc = [tc_box_net(m) for m in mlps]
    o_all, d_all = wl.camera_rays(64, 64)
    ro, rd = torch.from_numpy(o_all).to(dev), torch.from_numpy(d_all).to(dev)
    out = {"workload": "16 resident nets (12 of the uneven generator, seeds 1000..1011, + 4 ELU "
                       "39(PE)-[512]x6-1, seeds 2..5); Poisson arrivals (seed 5); 1/3 each: 64x64 "
                       "camera ray tile (affine-fixed, delta 1e-3, cap 200 iterations), U[256,65536] "
                       "boxes (affine-truncate K=16 FP32 / K=64 BF16-sound), leaf extraction to depth 9 "
                       "(K=16 FP32, 2^20-node leaf and per-level frontier buffers, wider levels walked in "
                       "chunks) on the 6 uneven nets whose depth-9 leaves fit 2^20 "
                       f"(indices {list(SERVING_LEAF_NETS)}); BF16-sound form (rays and boxes) for half "
                       "the requests whose net has that kernel",
           "slots": slots, "frontier_budget_bytes": budget, "rates": []}
    for lam in rates:
        rng = np.random.default_rng(5)
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=n_req))
        reqs, keep, meta = [], [], []
        for i in range(n_req):
            kind = int(rng.integers(0, 3))
            j = int(rng.integers(0, len(mlps)))
            bf = bool(rng.random() < 0.5)
            if kind == 0:
                form = 2 if (bf and ray_tc[j]) else 0
                t = torch.empty(ro.shape[0], dtype=torch.float32, device=dev)
                it = torch.empty(ro.shape[0], dtype=torch.int32, device=dev)
                keep.append((t, it))
                reqs.append(sra.ray_request(j, form, arrivals[i], ro, rd, t, it))
            elif kind == 1:
                n = int(rng.integers(256, 65537))
                c, h = wl.make_boxes(n, seed=300 + i)
                c, h = torch.from_numpy(c).to(dev), torch.from_numpy(h).to(dev)
                lo = torch.empty(n, dtype=torch.float32, device=dev)
                hi = torch.empty(n, dtype=torch.float32, device=dev)
                cl = torch.empty(n, dtype=torch.uint8, device=dev)
                keep.append((c, h, lo, hi, cl))
                form = 3 if (bf and box_tc[j]) else 1
                reqs.append(sra.box_request(j, form, arrivals[i], c, h, lo, hi, cl))
            else:
                leaves = torch.empty((1 << 20, 4), dtype=torch.int16, device=dev)
                keep.append(leaves)
                form = 1
                j = SERVING_LEAF_NETS[j % len(SERVING_LEAF_NETS)]
                reqs.append(sra.leaf_request(j, form, arrivals[i], 9, leaves))
            meta.append((kind, form))
        torch.cuda.synchronize()
        res = sra.serve(nets, forms, reqs, slots=slots, frontier_bytes=budget, realtime=True)
        lat = np.array([r.t_done - r.arrival for r in res]) * 1e3
        span = max(r.t_done for r in res) - min(r.arrival for r in res)
        st = np.array([r.status for r in res])
        per = {}
        for name, sel in (("rays", [m[0] == 0 for m in meta]), ("boxes", [m[0] == 1 for m in meta]),
                          ("leaves", [m[0] == 2 for m in meta]),
                          ("bf16_form", [m[1] in (2, 3) for m in meta]),
                          ("fp32_form", [m[1] in (0, 1) for m in meta])):
            sel = np.array(sel)
            if sel.any():
                per[name] = {"n": int(sel.sum()), "p50_ms": float(np.percentile(lat[sel], 50)),
                             "p99_ms": float(np.percentile(lat[sel], 99))}
        out["rates"].append({
            "offered_req_per_s": lam, "requests": n_req,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "throughput_req_per_s": n_req / span,
            "ok": int((st == 0).sum()), "capacity_exceeded": int((st == 5).sum()),
            "other_errors": int(((st != 0) & (st != 5)).sum()),
            "max_concurrent_slots_used": len({r.slot for r in res if r.slot >= 0}),
            "leaves_per_leaf_job": [int(r.n_out) for r, m in zip(res, meta) if m[0] == 2],
            "by": per})
        del keep
    for n in nets:
        n.close()
    return out


def batched_phase(sra, torch, cap):
    """64 uneven networks (widths 32..512, depths 3..10, ReLU / ELU / SIREN sin,
    octree depths 8..11; generator seeds 1000..1063): autotune K and the CTA
    shape per network, then build every tree level by level with one batched
    round per level (sra_classify_and_split_batch), against the same trees
    built one network and one level at a time."""
    from paper_2202_02444_gb300 import autotune, batch
    mlps = [wl.net_batch_mix(i) for i in range(64)]
    nets = [sra.Net(m) for m in mlps]
    depths = [int(m.meta["octree_depth"]) for m in mlps]
    t0 = time.perf_counter()
    tuned = [autotune.tune(n, m, d, probe_level=4, sample=2048, reps=2) for m, n, d in zip(mlps, nets, depths)]
    t_tune = time.perf_counter() - t0
    opts = [sra.make_opts(arith="truncate", K=r["K"], block_threads=r["block_threads"]) for r in tuned]
    batch.build_trees(nets[:4], opts[:4], [2] * 4, cap=cap)  # warm-up of the launch paths
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res, rounds = batch.build_trees(nets, opts, depths, cap=cap)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    t0 = time.perf_counter()
    res1 = batch.build_trees_one_by_one(nets, opts, depths, cap=cap)
    torch.cuda.synchronize()
    t1 = time.perf_counter() - t0
    nodes = sum(r["nodes"] for r in res)
    flop = sum(r["nodes"] * box_flops(m, t["K"]) for r, m, t in zip(res, mlps, tuned))
    same = all(a["levels"] == b["levels"] and a["leaves"] == b["leaves"] for a, b in zip(res, res1))
    # the same 64 trees with BF16-sound bounds on the tensor cores for every
    # network that has that kernel (one width 32, 64, 128, 256 or 512; K = 16,
    # 32, 64, or 128 below width 512), the others in their autotuned FP32
    # form, all in the same batched rounds
    tc = [tc_box_net(m) for m in mlps]
    # the tensor-core kernel's K: the autotuned one where it has a kernel for it, else 64
    k_tc = [r["K"] if r["K"] in (16, 32, 64) or (r["K"] == 128 and max(m.widths[1:-1]) <= 256) else 64
            for r, m in zip(tuned, mlps)]
    opts_tc = [sra.make_opts(arith="truncate", K=kt, precision="bf16_sound") if t else o
               for t, o, kt in zip(tc, opts, k_tc)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res_tc, rounds_tc = batch.build_trees(nets, opts_tc, depths, cap=cap)
    torch.cuda.synchronize()
    t_tc = time.perf_counter() - t0
    for n, t in zip(nets, tc):
        if t:
            sra.sync_status(n)
    nodes_tc = sum(r["nodes"] for r in res_tc)
    flop_tc = sum(r["nodes"] * box_flops(m, kt if t else u["K"]) for r, m, t, u, kt in zip(res_tc, mlps, tc, tuned, k_tc))
    ks_tc = {}
    for t, kt in zip(tc, k_tc):
        if t:
            ks_tc[str(kt)] = ks_tc.get(str(kt), 0) + 1
    bf16_sound = {"nets_on_tensor_cores": int(sum(tc)), "box_evals": nodes_tc, "rounds": rounds_tc, "s": t_tc,
                  "evals_per_s": nodes_tc / t_tc, "tflops": flop_tc / t_tc / 1e12,
                  "tensor_core_box_evals": int(sum(r["nodes"] for r, t in zip(res_tc, tc) if t)),
                  "tensor_core_K": ks_tc,
                  "nets_truncated_at_cap": int(sum(r["truncated"] for r in res_tc)),
                  "tensor_core_nets_truncated_at_cap": int(sum(r["truncated"] for r, t in zip(res_tc, tc) if t))}
    for n in nets:
        n.close()
    ks = {}
    for t in tuned:
        ks[str(t["K"])] = ks.get(str(t["K"]), 0) + 1
    return {"workload": "64 nets of the uneven generator (seeds 1000..1063): width U{32..512}, depth "
                        "U[3,10], ReLU/ELU/SIREN-sin, octree depth U[8,11]; affine-truncate FP32 with K and "
                        f"threads per CTA autotuned per net; frontier cap {cap} nodes per net per level",
            "box_evals": nodes, "rounds": rounds,
            "batched_s": tb, "batched_evals_per_s": nodes / tb, "batched_tflops": flop / tb / 1e12,
            "one_by_one_s": t1, "one_by_one_evals_per_s": nodes / t1,
            "batched_vs_one_by_one": t1 / tb, "same_trees": same,
            "nets_truncated_at_cap": int(sum(r["truncated"] for r in res)),
            "autotune_s": t_tune, "autotune_K": ks, "bf16_sound_where_served": bf16_sound,
            "wall_clock_note": "host-timed with synchronisation (one counter read per level)"}


def policies_phase(sra, torch, dev):
    """The range-analysis policies of Sec. 3 side by side on the paper's
    8-layer 32-wide architecture (ReLU 3-[32]x7-1, He init, seed 41; the
    trained shapes of its Table 1 are not available): 65,536 boxes with
    half-widths log-uniform in [1/256, 1/20], FP32. Cost is reported per box
    and relative to a plain forward evaluation of one point (sra_eval), the
    normalisation of Table 1; width is the mean output range."""
    mlp = wl.make_mlp([32] * 7, "relu", seed=41)
    net = sra.Net(mlp)
    B = 1 << 16
    c, h = wl.make_boxes(B, seed=1, hw_lo=1 / 256, hw_hi=1 / 20)
    C_, H_ = torch.from_numpy(c).to(dev), torch.from_numpy(h).to(dev)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r = fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts), r

    ev_ms, _ = timed(lambda: sra.evaluate(net, C_))
    res = {"workload": "ReLU 3-[32]x7-1 (He init, seed 41), 65,536 boxes, half-widths log-U[1/256, 1/20], FP32",
           "forward_evals_per_s": B / (ev_ms / 1e3), "policies": {}}
    for name, arith, K in (("interval", "interval", 0), ("affine-fixed", "fixed", 0),
                           ("affine-truncate K=16", "truncate", 16), ("affine-truncate K=64", "truncate", 64),
                           ("affine-full", "full", 0)):
        o = sra.make_opts(arith=arith, K=K)
        ms, (lo, hi, cl) = timed(lambda: sra.bound_boxes(net, C_, H_, opts=o))
        res["policies"][name] = {"box_evals_per_s": B / (ms / 1e3), "cost_vs_forward": ms / ev_ms,
                                 "mean_width": float((hi - lo).mean()),
                                 "unknown_frac": float((cl == 0).float().mean())}
    res["paper_table1_3d_cost_vs_forward"] = {"interval": 2.3, "affine-fixed": 6.7, "affine-truncate": 69.0,
                                              "affine-full": 96.4, "hardware": "RTX 2070, JAX"}
    net.close()
    # the config-2 network: affine-full keeps 2051 symbols, each box's noise
    # matrix in device memory (one batched GEMM per layer)
    wide = wl.net_relu256x8()
    net = sra.Net(wide)
    Bw = 4096
    c, h = wl.make_boxes(Bw, seed=1, hw_lo=1 / 1024, hw_hi=1 / 64)
    C_, H_ = torch.from_numpy(c).to(dev), torch.from_numpy(h).to(dev)
    res["wide"] = {"workload": f"ReLU 3-[256]x8-1 (seed 1), {Bw} boxes, half-widths log-U[1/1024, 1/64], FP32",
                   "policies": {}}
    for name, arith, K in (("affine-truncate K=64", "truncate", 64), ("affine-full", "full", 0)):
        o = sra.make_opts(arith=arith, K=K)
        ms, (lo, hi, cl) = timed(lambda: sra.bound_boxes(net, C_, H_, opts=o))
        flop = full_flops(wide) if arith == "full" else box_flops(wide, K)
        res["wide"]["policies"][name] = {"box_evals_per_s": Bw / (ms / 1e3), "mean_width": float((hi - lo).mean()),
                                         "unknown_frac": float((cl == 0).float().mean()),
                                         "flop_per_box": flop, "tflops": flop * Bw / (ms / 1e3) / 1e12}
    net.close()
    res["tc_widths"] = tc_widths_phase(sra, torch, dev, timed)
    return res


def tc_widths_phase(sra, torch, dev, timed):
    """The tensor-core bound kernel at each width it serves (3-[H]x4-1 ReLU,
    He init, seed 51; H = 64 runs the 128-wide kernel on zero-padded weights;
    H = 64, 128 and 256 bound two boxes per CTA, H = 512 one),
    affine-truncate K = 64 on 32,768 boxes (half-widths log-U[1/1024, 1/64]),
    against the FP32 SIMT kernel on the same boxes."""
    B = 1 << 15
    c, h = wl.make_boxes(B, seed=3, hw_lo=1 / 1024, hw_hi=1 / 64)
    C_, H_ = torch.from_numpy(c).to(dev), torch.from_numpy(h).to(dev)
    peak = measured_peak("bf16_tflops", 1900.0)[0]
    out = {"workload": f"ReLU 3-[H]x4-1 (He init, seed 51), {B} boxes, half-widths log-U[1/1024, 1/64], "
                       "affine-truncate K=64", "peak_tflops": peak, "widths": {}}
    for H in (64, 128, 256, 512):  # width 64 runs the 128-wide kernel on zero-padded weights
        mlp = wl.make_mlp([H] * 4, "relu", seed=51)
        net = sra.Net(mlp)
        flop = box_flops(mlp, 64)
        row = {"flop_per_box": flop}
        for prec in ("fp32", "bf16", "bf16_sound"):
            o = sra.make_opts(arith="truncate", K=64, precision=prec)
            try:
                ms, (lo, hi, cl) = timed(lambda: sra.bound_boxes(net, C_, H_, opts=o))
            except sra.SraError as e:  # the SIMT engine's per-box thread budget
                row[prec] = {"unsupported": str(e)}
                continue
            if prec != "fp32":
                sra.sync_status(net)
            tf = flop * B / (ms / 1e3) / 1e12
            row[prec] = {"box_evals_per_s": B / (ms / 1e3), "tflops": tf,
                         "frac_of_bf16_peak": tf / peak if prec != "fp32" else None,
                         "unknown_frac": float((cl == 0).float().mean())}
        if H == 256:  # the other kept-symbol counts of the kernel
            row["bf16_sound_by_K"] = {}
            for K in (16, 32, 128):
                o = sra.make_opts(arith="truncate", K=K, precision="bf16_sound")
                ms, (lo, hi, cl) = timed(lambda: sra.bound_boxes(net, C_, H_, opts=o))
                sra.sync_status(net)
                fk = box_flops(mlp, K)
                row["bf16_sound_by_K"][str(K)] = {"box_evals_per_s": B / (ms / 1e3), "flop_per_box": fk,
                                                  "tflops": fk * B / (ms / 1e3) / 1e12,
                                                  "frac_of_bf16_peak": fk * B / (ms / 1e3) / 1e12 / peak}
        out["widths"][str(H)] = row
        net.close()
    return out


def octree_phase(sra, torch, dev, net, depth=10, level_cap=1 << 21, K=64):
    """The whole octree of the 3-[256]x8-1 ReLU net to depth 10 (Proc. 3),
    level by level from the root, in FP32, and in plain BF16 and BF16-sound
    (tensor cores) with the FP64 re-check: each level's frontier is bounded in chunks of at most
    `level_cap` nodes (one sra_classify_and_split call each); a level whose
    frontier exceeds `level_cap` nodes ends the build. Per level: the frontier,
    the class counts and the device time of its rounds (CUDA events)."""
    forms = {"fp32": sra.make_opts(arith="truncate", K=K),
             "bf16": sra.make_opts(arith="truncate", K=K, precision="bf16", recheck=True, recheck_band=1e-5),
             "bf16_sound": sra.make_opts(arith="truncate", K=K, precision="bf16_sound", recheck=True,
                                         recheck_band=1e-5)}
    out = {"workload": f"octree of ReLU 3-[256]x8-1 (seed 1) over [-1,1]^3 to depth {depth}, affine-truncate "
                       f"K={K}; a level's frontier is bounded in chunks and may hold at most {level_cap} nodes",
           "forms": {}}
    buf = [torch.empty((8 * level_cap, 4), dtype=torch.int16, device=dev) for _ in range(2)]
    leaves = torch.empty((level_cap, 4), dtype=torch.int16, device=dev)
    counts = torch.zeros(8, dtype=torch.int64, device=dev)
    for name, o in forms.items():
        fr = sra.nodes_to_tensor(wl.root_node(), device=dev)
        levels, total_ms, evals, stop = [], 0.0, 0, None
        for level in range(depth + 1):
            n = fr.shape[0]
            if n == 0:
                break
            if n > level_cap:
                stop = f"level {level} frontier of {n} nodes exceeds {level_cap}"
                break
            nxt = buf[level % 2]
            counts.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sra.classify_and_split(net, fr, depth, opts=o, out=nxt, leaves=leaves, counts=counts)
            e1.record()
            torch.cuda.synchronize()
            sra.sync_status(net)
            ms = e0.elapsed_time(e1)
            c = counts.cpu().numpy()
            total_ms += ms
            evals += n
            levels.append({"level": level, "frontier": n, "pos": int(c[2]), "neg": int(c[3]), "unk": int(c[4]),
                           "leaves": int(c[1]), "rechecked": int(c[5]), "ms": ms})
            kids = int(c[0])
            fr = nxt[:min(kids, nxt.shape[0])]
            if kids > nxt.shape[0]:
                stop = f"level {level + 1} frontier of {kids} nodes exceeds {nxt.shape[0]}"
                break
        out["forms"][name] = {"levels": levels, "box_evals": evals, "device_ms": total_ms,
                              "box_evals_per_s": evals / (total_ms / 1e3) if total_ms > 0 else None,
                              "completed": stop is None, "stopped": stop,
                              "leaves_at_depth": levels[-1]["leaves"] if stop is None and levels else None}
    return out


def make_frontier(sra, net, level, batch, opts):
    """Children of the UNKNOWN nodes at `level - 1` of the network's octree
    (the real frontier the level visits), tiled to `batch` nodes."""
    import torch
    leaves, _ = sra.extract_leaves(net, level - 1, opts=opts)
    kids, _, cnt = sra.classify_and_split(net, leaves, level, opts=opts)
    torch.cuda.synchronize()
    nk = int(cnt[sra.CNT_CHILDREN])
    kids = kids[:nk]
    reps = (batch + nk - 1) // max(nk, 1)
    fr = kids.repeat(reps, 1)[:batch].contiguous()
    return fr, nk


def cpu_baseline(mlp, fr_nodes, K, nsample, nsample_1core):
    """The FP64 oracle on a bounded sample of the same frontier, on all host
    cores and, on a smaller sample, on one core."""
    import oracle
    onet = oracle.OracleNet(mlp)

    def timed(n, threads):
        nodes = fr_nodes[wl.sample_rows(len(fr_nodes), n, seed=5)]
        t0 = time.perf_counter()
        oracle.classify_nodes(onet, nodes, (-1, -1, -1), (1, 1, 1), oracle.OCTREE, "truncate", K=K,
                              nthreads=threads)
        return len(nodes), time.perf_counter() - t0

    n_all, dt = timed(nsample, 0)
    line = {"value": n_all / dt, "unit": "box-bound evals/s", "cores": oracle.max_threads(),
            "kind": "oracle",
            "sample": f"{n_all} level-7 frontier nodes of the 3-[256]x8-1 ReLU net, "
                      f"affine-truncate K={K}, FP64, {dt:.1f} s"}
    if nsample_1core > 0:
        n1, dt1 = timed(nsample_1core, 1)
        line["single_core"] = {"value": n1 / dt1, "unit": "box-bound evals/s", "cores": 1,
                               "sample": f"{n1} nodes of the same frontier, {dt1:.1f} s"}
    return line


def cpu_baseline_rays(mlp, o, d, nrays=32, iters=200):
    """The FP64 oracle's CastRay (Proc. 2) on a bounded sample of the camera
    tile's rays (each capped at `iters` iterations), on all host cores:
    ray-iterations/s, the unit the rays' rate is built from."""
    import oracle
    onet = oracle.OracleNet(mlp)
    t0 = time.perf_counter()
    r = oracle.cast_rays(onet, o[:nrays], d[:nrays], "fixed", delta=1e-4, t_max=10.0, sigma0=1.0,
                         max_iters=iters)
    dt = time.perf_counter() - t0
    n_it = int(np.sum(r["iters"]))
    return {"value": n_it / dt, "unit": "ray-iterations/s", "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{nrays} central camera rays of the 39(PE)-[512]x6-1 ELU net, affine-fixed FP64, "
                      f"{iters} iterations each at most ({n_it} in all), {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    mlp = wl.net_relu256x8()
    K = 64
    rng = np.random.default_rng(1)
    # the GPU arm's frontier needs the network's own level-6 tree, which the
    # oracle cannot build in minutes; uniformly drawn level-7 nodes cost the
    # same per box (the bound's work does not depend on where the box is)
    nodes = wl.random_nodes(args.ref_sample, level=args.frontier_level, seed=int(rng.integers(1 << 30)))
    onet = oracle.OracleNet(mlp)
    for _ in range(args.warmup):
        oracle.classify_nodes(onet, nodes[:4], (-1, -1, -1), (1, 1, 1), oracle.OCTREE, "truncate", K=K)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.classify_nodes(onet, nodes, (-1, -1, -1), (1, 1, 1), oracle.OCTREE, "truncate", K=K)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = len(nodes) / (ms / 1e3)
    line = {"impl": "reference", "metric": "box-bound evals/s", "value": value,
            "unit": "box-bound evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "octree round of ReLU 3-[256]x8-1, affine-truncate K=64 "
                                   f"(sample of {len(nodes)} level-{args.frontier_level} nodes per step)"},
            "cpu_baseline": {"value": value, "unit": "box-bound evals/s", "cores": oracle.max_threads(),
                             "kind": "oracle", "sample": f"{len(nodes)} nodes per step"},
            "e2e": {"value": value, "unit": "box-bound evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def kernel_case(args):
    """The dominant kernel alone, for profilers: two sra_bound_boxes calls on
    --batch boxes (half-widths log-uniform in [1/1024, 1/64]) of the
    3-[256]x8-1 ReLU net, affine-truncate K=64 in the given precision, or
    affine-full in FP32 (full_fp32), or BF16-sound on the 3-[512]x4-1 ReLU
    net (bf16_sound_512), or BF16-sound with K=16 on the 3-[256]x4-1 ReLU net
    (bf16_sound_k16)."""
    import torch
    from paper_2202_02444_gb300 import sra
    if args.kernel_case in ("rays", "rays_bf16"):  # central camera rays, 300-iteration cap
        net = sra.Net(wl.net_elu512x6_pe())
        o, d = wl.camera_rays(1920, 1080)
        side = 8 if args.kernel_case == "rays" else 32
        sel = np.array([(540 - side // 2 + j) * 1920 + 960 - side // 2 + i
                        for j in range(side) for i in range(side)])
        ro, rd = torch.from_numpy(o[sel]).cuda(), torch.from_numpy(d[sel]).cuda()
        prec = "bf16" if args.kernel_case == "rays_bf16" else "fp32"
        ropts = sra.make_opts(arith="fixed", delta=1e-4, t_max=10.0, max_iters=300, precision=prec)
        for _ in range(2):
            sra.cast_rays(net, ro, rd, opts=ropts)
        torch.cuda.synchronize()
        print("kernel case done rays")
        return
    wide = args.kernel_case == "bf16_sound_512"  # the width-512 net of policies.tc_widths
    k16 = args.kernel_case == "bf16_sound_k16"  # the width-256 net of policies.tc_widths at K = 16
    net = sra.Net(wl.make_mlp([512 if wide else 256] * 4, "relu", seed=51) if (wide or k16) else wl.net_relu256x8())
    c, h = wl.make_boxes(args.batch, seed=1, hw_lo=1 / 1024, hw_hi=1 / 64)
    C_, H_ = torch.from_numpy(c).cuda(), torch.from_numpy(h).cuda()
    if args.kernel_case == "full_fp32":  # affine-full, the noise matrix in device memory
        o = sra.make_opts(arith="full")
    elif wide or k16:
        o = sra.make_opts(arith="truncate", K=16 if k16 else 64, precision="bf16_sound")
    else:
        o = sra.make_opts(arith="truncate", K=64, precision=args.kernel_case)
    for _ in range(2):
        sra.bound_boxes(net, C_, H_, opts=o)
    torch.cuda.synchronize()
    print("kernel case done", args.kernel_case, args.batch)


def free_port():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def spawn_ranks(args):
    """--gpus N > 1 started without a launcher: run this script again under
    torch.distributed.run with N local ranks (one per GPU) and return its exit
    code; None when there is nothing to spawn."""
    if args.gpus <= 1 or "WORLD_SIZE" in os.environ:
        return None
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), os.path.abspath(__file__),
           *sys.argv[1:]]
    return subprocess.call(cmd)


def main():
    args = parse_args()
    rc = spawn_ranks(args)
    if rc is not None:
        sys.exit(rc)
    if args.kernel_case:
        kernel_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2202_02444_gb300 import sra

    dev = torch.device("cuda", local)
    K = 64
    mlp_box = wl.net_relu256x8()
    mlp_ray = wl.net_elu512x6_pe()
    net_box = sra.Net(mlp_box)
    net_ray = sra.Net(mlp_ray)
    bopts = sra.make_opts(arith="truncate", K=K, precision=args.precision, recheck=True,
                          recheck_band=1e-5)
    # weak scaling: each rank owns its own frontier batch and ray tile
    # the frontier (a bench input) comes from the FP32 octree of the network
    fr_all, n_real = make_frontier(sra, net_box, args.frontier_level, args.batch * world,
                                   sra.make_opts(arith="truncate", K=K))
    fr = rank_batch(fr_all, args.batch, rank).contiguous()  # this rank's batch of the global frontier
    B = fr.shape[0]
    o, d = wl.camera_rays(1920, 1080)
    T = args.ray_tile
    sel = np.array(rank_ray_tile(1920, 1080, T, rank))
    ro = torch.from_numpy(o[sel]).to(dev)
    rd = torch.from_numpy(d[sel]).to(dev)
    R = len(sel)
    out = torch.empty((8 * B, 4), dtype=torch.int16, device=dev)
    leaves = torch.empty((B, 4), dtype=torch.int16, device=dev)
    counts = torch.zeros(8, dtype=torch.int64, device=dev)
    t_hit = torch.empty(R, dtype=torch.float32, device=dev)
    iters = torch.empty(R, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def step_boxes():
        counts.zero_()
        sra.classify_and_split(net_box, fr, args.frontier_level + 3, opts=bopts, out=out,
                               leaves=leaves, counts=counts)

    for _ in range(args.warmup):
        step_boxes()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with ClockSampler(local, enabled=not args.no_clocks) as clk:
        torch.cuda.nvtx.range_push("timed_steps")  # profilers filter on this range
        for k in range(args.steps):
            flush.zero_()  # evict L2 between steps (outside the events)
            a, b = ev[k]
            a.record()
            step_boxes()
            b.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    box_ms = [a.elapsed_time(b) for a, b in ev]
    cnt = counts.cpu().numpy()

    # the bound kernel alone, in each form, over the same boxes
    nodes_h = sra.tensor_to_nodes(fr)
    w = 2.0 / (1 << nodes_h["level"].astype(np.int64))
    lo_ = -1.0 + np.stack([nodes_h["ix"], nodes_h["iy"], nodes_h["iz"]], 1) * w[:, None]
    cen = torch.from_numpy((lo_ + 0.5 * w[:, None]).astype(np.float32)).to(dev)
    hw = torch.from_numpy(np.repeat((0.5 * w)[:, None], 3, 1).astype(np.float32)).to(dev)
    blo = torch.empty(B, dtype=torch.float32, device=dev)
    bhi = torch.empty(B, dtype=torch.float32, device=dev)
    bcl = torch.empty(B, dtype=torch.uint8, device=dev)
    forms = {}
    for prec in ("fp32", "bf16", "bf16_sound"):
        kopts = sra.make_opts(arith="truncate", K=K, precision=prec)
        sra.bound_boxes(net_box, cen, hw, opts=kopts, lo=blo, hi=bhi, cls=bcl)
        kb = []
        for k in range(3):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sra.bound_boxes(net_box, cen, hw, opts=kopts, lo=blo, hi=bhi, cls=bcl)
            e1.record()
            torch.cuda.synchronize()
            kb.append(e0.elapsed_time(e1))
        ms = statistics.median(kb)
        cl = bcl.cpu().numpy()
        forms[prec] = {"box_evals_per_s": B / (ms / 1e3), "kernel_ms": ms,
                       "unknown_frac": float((cl == 0).mean())}
    kern_ms = forms[args.precision]["kernel_ms"]

    # end to end through the public API with host buffers
    fr_host = fr.cpu().pin_memory()
    out_host = torch.empty((8 * B, 4), dtype=torch.int16).pin_memory()
    cnt_host = torch.empty(8, dtype=torch.int64).pin_memory()
    e2e_t, d2h_list = [], []
    h2d = fr_host.numel() * 2
    for k in range(max(2, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fr_dev = fr_host.to(dev, non_blocking=True)
        counts.zero_()
        sra.classify_and_split(net_box, fr_dev, args.frontier_level + 3, opts=bopts, out=out,
                               leaves=leaves, counts=counts)
        cnt_host.copy_(counts, non_blocking=True)
        torch.cuda.synchronize()
        nch = int(cnt_host[0])
        out_host[:nch].copy_(out[:nch])
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
        d2h_list.append(cnt_host.numel() * 8 + nch * 8)

    # ray phase (separate from the step): a camera tile with an iteration cap,
    # in each form: FP32 on the SIMT cores, split-BF16 hidden layers on tcgen05
    # (plain, and BF16-sound: segment bounds with the a-priori rounding
    # radius), and the BF16 forms with the FP64 re-check of rays that met a
    # near-zero decision
    ray_forms, ray_t = {}, {}
    it_flop = ray_iter_flops(mlp_ray)
    rechecked = torch.zeros(1, dtype=torch.int64, device=dev)
    for form in ("fp32", "bf16", "bf16_fp64_recheck", "bf16_sound", "bf16_sound_fp64_recheck"):
        prec = form.replace("_fp64_recheck", "")
        ropts = sra.make_opts(arith="fixed", delta=1e-4, t_max=10.0, max_iters=args.ray_iters,
                              precision=prec, recheck=form.endswith("recheck"), recheck_band=1e-5,
                              recheck_count=rechecked)
        sra.cast_rays(net_ray, ro[:64], rd[:64], opts=ropts)
        torch.cuda.synchronize()
        rechecked.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sra.cast_rays(net_ray, ro, rd, opts=ropts, t_hit=t_hit, iters=iters)
        e1.record()
        torch.cuda.synchronize()
        sra.sync_status(net_ray)
        ray_ms = e0.elapsed_time(e1)
        iters_h = iters.cpu().numpy()
        t_h = t_hit.cpu().numpy()
        done = ~np.isnan(t_h)
        ray_t[form] = t_h
        ray_forms[form] = {
            "ms": ray_ms, "rays": R, "completed": int(done.sum()),
            "rays_per_s": float(done.sum()) / (ray_ms / 1e3),
            "ray_iters_per_s": float(iters_h.sum()) / (ray_ms / 1e3),
            "tflops": float(iters_h.sum()) * it_flop / (ray_ms / 1e3) / 1e12,
            "iters_mean": float(iters_h.mean()), "iters_max": int(iters_h.max()),
            "hits": int(np.isfinite(t_h).sum())}
        if form.endswith("recheck"):
            ray_forms[form]["rays_rechecked_fp64"] = int(rechecked.item())
            ray_forms[form]["recheck_band"] = 1e-5
    # completion sample: the central 96x96 pixels (9216 rays, about four
    # waves of the tensor-core kernel's 16 ray slots per SM, so slots refill
    # as rays end) marched to the end; rays/s of each form is its measured
    # iteration rate over the sample's mean iterations per ray
    completion = None
    if args.ray_complete_cap > 0:
        csel = np.array(rank_ray_tile(1920, 1080, 96, rank))
        nc = len(csel)
        slots = 16 * torch.cuda.get_device_properties(dev).multi_processor_count
        cro, crd = torch.from_numpy(o[csel]).to(dev), torch.from_numpy(d[csel]).to(dev)
        copts = sra.make_opts(arith="fixed", delta=1e-4, t_max=10.0, max_iters=args.ray_complete_cap,
                              precision="bf16_sound")
        tc_ = torch.empty(nc, dtype=torch.float32, device=dev)
        ic_ = torch.empty(nc, dtype=torch.int32, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sra.cast_rays(net_ray, cro, crd, opts=copts, t_hit=tc_, iters=ic_)
        e1.record()
        torch.cuda.synchronize()
        sra.sync_status(net_ray)
        c_ms = e0.elapsed_time(e1)
        t_c, i_c = tc_.cpu().numpy(), ic_.cpu().numpy()
        ended = ~np.isnan(t_c)
        it_mean = float(i_c[ended].mean()) if ended.any() else float("nan")
        completion = {"rays": int(nc), "waves": nc / slots, "form": "bf16_sound", "cap": args.ray_complete_cap,
                      "ms": c_ms,
                      "completed": int(ended.sum()), "hits": int(np.isfinite(t_c).sum()),
                      "rays_per_s": float(ended.sum()) / (c_ms / 1e3),
                      "iters_per_completed_ray": it_mean,
                      "frame_fraction": nc / (1920 * 1080),
                      "frame_estimate_s": (1920 * 1080) / max(float(ended.sum()) / (c_ms / 1e3), 1e-30),
                      "frame_note": "the 1920x1080 frame (2,073,600 rays) at this sample's completed-ray rate; "
                                    "the sample is the central 96x96 pixels, about four waves of ray slots"}
        for form, rf in ray_forms.items():
            rf["rays_per_s_at_sample_iters"] = rf["ray_iters_per_s"] / it_mean if ended.any() else None
    ta, tb = ray_t["fp32"], ray_t["bf16"]
    fin = np.isfinite(ta) & np.isfinite(tb)
    agree = (np.isfinite(ta) == np.isfinite(tb)) & (np.isnan(ta) == np.isnan(tb))
    agree[fin] &= np.abs(ta[fin] - tb[fin]) <= 1e-4 * 1.0001 + 1e-6

    # mesh phase: hierarchical mesh extraction (Sec. 4.7) of the ReLU
    # 3-32-32-1 network (the 256x8 network is negative everywhere in the root
    # box: it has no surface): UNKNOWN leaves at depth 7, then 8^3 sub-cells per
    # leaf (1024^3 effective grid), marching tetrahedra
    mesh = None
    if rank == 0:
        net_small = sra.Net(wl.net_small_relu())
        mo = sra.make_opts(arith="fixed")
        sra.mesh_leaves(net_small, sra.extract_leaves(net_small, 3, opts=mo)[0], 3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ml, _ = sra.extract_leaves(net_small, 7, opts=mo)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        tris = sra.mesh_leaves(net_small, ml, 3)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        nl = int(ml.shape[0])
        mesh = {"workload": "ReLU 3-32-32-1 (seed 0): UNKNOWN leaves of its depth-7 octree (affine-fixed), "
                            "8^3 sub-cells per leaf (1024^3 effective grid), marching tetrahedra",
                "leaves": nl, "leaf_fraction": nl / 8 ** 7, "triangles": int(tris.shape[0]),
                "tree_s": t1 - t0, "mesh_s": t2 - t1, "leaves_per_s": nl / (t2 - t1),
                "point_evals_per_s": nl * 729 / (t2 - t1),
                "timing": "host clock around the synchronous calls"}
        del tris
        net_small.close()

    # frustum ray casting (Sec. 4.3) against per-pixel CastRay, 512x512 image of
    # an ELU 3-[128]x4-1 network with a surface in view (seed 23: half of the
    # root box negative)
    frustum = None
    if rank == 0:
        net_small = sra.Net(wl.make_mlp([128] * 4, "elu", seed=23))
        Wf = Hf = 512
        of, df = wl.camera_rays(Wf, Hf)
        dft, oft = torch.from_numpy(df).to(dev), torch.from_numpy(of).to(dev)
        fo = sra.make_opts(arith="fixed", delta=1e-3, max_iters=1 << 16)
        sra.cast_frustum(net_small, of[0], dft[:64 * 64], 64, 64, opts=fo)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tf_, itf, fst = sra.cast_frustum(net_small, of[0], dft, Wf, Hf, grid=16, opts=fo)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        tr_, itr = sra.cast_rays(net_small, oft, dft, opts=fo)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        a_, b_ = tf_.cpu().numpy(), tr_.cpu().numpy()
        fa, fb = np.isfinite(a_), np.isfinite(b_)
        agree = (fa == fb)
        agree[fa & fb] &= np.abs(a_[fa & fb] - b_[fa & fb]) <= 1e-3 * 1.0001 + 1e-6
        npx = Wf * Hf
        frustum = {"workload": "512x512 camera at (0,0,3) vs ELU 3-[128]x4-1 (He init, seed 23), affine-fixed "
                               "FP32, delta 1e-3, 16x16 coarse frusta",
                   "frustum_s": t1 - t0, "per_ray_s": t2 - t1,
                   "frustum_steps_per_pixel": (fst["frustum_boxes"] + int(itf.sum())) / npx,
                   "per_ray_steps_per_pixel": int(itr.sum()) / npx,
                   "rounds": fst["rounds"], "pixels_handed_to_rays": fst["rays"],
                   "same_as_per_ray_frac": float(agree.mean()), "hits": int(fa.sum()),
                   "timing": "host clock around synchronous calls (the frustum march reads a count per round)"}
        net_small.close()

    # empty-sphere queries (Sec. 4.4) on the same network
    spheres = None
    if rank == 0:
        qp = torch.from_numpy(np.random.default_rng(9).uniform(-1, 1, (1 << 16, 3)).astype(np.float32)).to(dev)
        so = sra.make_opts(arith="truncate", K=K)
        sra.empty_spheres(net_box, qp[:256], 1.0, 12, opts=so)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rad = sra.empty_spheres(net_box, qp, 1.0, 12, opts=so)
        e1.record()
        torch.cuda.synchronize()
        sms = e0.elapsed_time(e1)
        spheres = {"workload": "65,536 uniform points in [-1,1]^3, ReLU 3-[256]x8-1, affine-truncate K=64 FP32, "
                               "boxes of half-width 2^-k, k < 12",
                   "ms": sms, "queries_per_s": (1 << 16) / (sms / 1e3),
                   "decided_frac": float((rad > 0).float().mean()), "median_radius": float(rad.median())}

    policies = policies_phase(sra, torch, dev) if rank == 0 else None
    octree = octree_phase(sra, torch, dev, net_box) if rank == 0 and not args.no_octree else None

    batched = None
    if not args.no_batched and rank == 0:
        batched = batched_phase(sra, torch, args.batched_cap)
    serving = None
    if not args.no_serve and rank == 0:
        rates = [float(x) for x in args.serve_rates.split(",") if x]
        serving = serving_phase(sra, torch, dev, rates, args.serve_requests)

    mean_box = statistics.mean(box_ms)
    t_local = torch.tensor([mean_box], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
    mean_box = float(t_local[0])
    value = world * B / (mean_box / 1e3)
    flop_box = box_flops(mlp_box, K)
    # the bound kernel's launch duration inside the timed steps: each step is
    # one sra_classify_and_split call, bracketed by CUDA events on the stream
    # the kernel runs on; the bound kernel is > 98 % of a step (launch list),
    # so the step time is a slight over-estimate of the launch duration
    achieved = flop_box * B / (mean_box / 1e3) / 1e12
    clocks = clk.summary()
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    if args.precision == "fp32":
        peak, bound, kname = 152 * 128 * 2 * sm_max * 1e6 / 1e12, "alu", "bound_kernel<float,64> (FP32 FFMA)"
        peak_src = "152 SMs x 128 FP32 lanes x 2 flop x max SM clock"
    else:
        peak, bound = measured_peak("bf16_tflops", 1900.0)
        kname = f"tc_bound_kernel<256,{'true' if args.precision == 'bf16_sound' else 'false'},ReLU> (tcgen05 BF16)"
        peak_src = "MEASURED_PEAKS.json bf16_tflops (burst, cuBLAS) of measured"
        bound = "tensor"
    if rank == 0:
        try:
            cpu = cpu_baseline(mlp_box, nodes_h[:max(1, min(B, n_real))], K, args.cpu_sample,
                               args.cpu_sample_1core)
        except Exception as e:  # noqa: BLE001 - reported, not fatal
            cpu = {"value": None, "error": str(e)[:200]}
        try:
            cpu_rays = cpu_baseline_rays(mlp_ray, o[sel].astype(np.float64), d[sel].astype(np.float64))
        except Exception as e:  # noqa: BLE001 - reported, not fatal
            cpu_rays = {"value": None, "error": str(e)[:200]}
        line = {
            "metric": "box-bound evals/s", "value": value, "unit": "box-bound evals/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": mean_box, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "bf16",
            "precision": args.precision,
            "data": "synthetic",
            "config": {"workload": f"octree round of ReLU 3-[256]x8-1 (He init, seed 1), "
                                   f"affine-truncate K={K}, {args.precision}, FP64 re-check band 1e-5, "
                                   f"{B} level-{args.frontier_level} frontier nodes per step",
                       "frontier_nodes": B, "distinct_frontier_nodes": n_real,
                       "l2": "flushed between steps (256 MB write)"},
            "frontier_counts": {"pos": int(cnt[2]), "neg": int(cnt[3]), "unk": int(cnt[4]),
                                "children": int(cnt[0]), "rechecked": int(cnt[5])},
            "e2e": {"value": world * B / statistics.median(e2e_t), "unit": "box-bound evals/s",
                    "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(statistics.median(d2h_list))},
            "gpu_launches": args.steps * 5,
            "roofline": {"bound": bound, "kernel": kname,
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "traffic": captured_traffic("tc_bound_kernel<256,true,ReLU>")
                         if args.precision == "bf16_sound" else None,
                         "kernel_ms": mean_box, "kernel_ms_alone": kern_ms,
                         "timing": "CUDA events around each timed step (bound kernel + compaction)",
                         "flop_per_box": flop_box,
                         "peak_source": peak_src},
            "forms": forms,
            "rays": {"workload": f"{T}x{T} central pixels of a 1920x1080 camera at (0,0,3) vs ELU "
                                 f"39(PE 6 octaves)-[512]x6-1, affine-fixed, delta 1e-4, t_max 10, "
                                 f"cap {args.ray_iters} iterations per ray",
                     "flop_per_iter": it_flop, "forms": ray_forms, "completion_sample": completion,
                     "same_outcome_frac": float(agree.mean()),
                     "bf16_vs_fp32_iters_per_s": ray_forms["bf16"]["ray_iters_per_s"]
                     / max(ray_forms["fp32"]["ray_iters_per_s"], 1e-30),
                     "cpu_baseline": cpu_rays},
            "mesh": mesh,
            "empty_spheres": spheres,
            "frustum": frustum,
            "policies": policies,
            "octree_depth10": octree,
            "batched": batched,
            "serving": serving,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "wall_s": wall,
        }
        print(json.dumps(line), flush=True)
    net_box.close()
    net_ray.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
