"""What the segment bounds of CastRay decide on the 39(PE)-[512]x6-1 ELU
network (the 1920x1080 ray-casting workload), from the oracle alone.

Proc. 2 advances by max(0.98 sigma*, delta) per iteration, where sigma* is
the length of the last segment whose bound decided a sign (0 when it stayed
UNKNOWN). Every one of the 64 golden rays (tests/golden/, the oracle's
CastRay, delta 1e-4) took exactly round(t_hit / delta) + 1 iterations: no
segment bound along any of them decided a sign, so on this random-init
network the march samples f every delta. Segments of length 1e-4 to 1e-2
just before each hit stay UNKNOWN in the oracle's FP64 affine-fixed bound.

A guaranteed (rounding-aware) bound contains the exact-arithmetic one, so it
cannot decide a segment that the exact bound leaves UNKNOWN: on this workload
a rounding radius on the tensor-core ray kernel would change no decision, and
the kernel carries none (its BF16 decisions near zero go to the FP64
re-check instead).
"""
import json
import os

import numpy as np

import oracle
from paper_2202_02444_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "camera_rays_elu512x6_pe.json")


def golden():
    g = json.load(open(GOLDEN))
    return g, np.array([float(x) for x in g["t"]]), np.array(g["iters"])


def test_golden_rays_step_by_delta_only():
    g, t, it = golden()
    assert np.all(np.array(g["status"]) == 1)
    # t after k UNKNOWN steps is k * delta (the step is delta when sigma* = 0)
    assert np.array_equal(it, np.round(t / g["delta"]).astype(np.int64) + 1)


def test_segments_before_the_hits_stay_unknown():
    g, t, _ = golden()
    mlp = oracle.OracleNet(wl.net_elu512x6_pe())
    o, d = wl.camera_rays(g["camera"]["width"], g["camera"]["height"])
    sel = np.array(g["pixels"])[::4]  # 16 of the 64 rays
    th = t[::4]
    for sigma in (1e-4, 1e-3, 1e-2):
        for p, r, tk in zip(o[sel].astype(np.float64), d[sel].astype(np.float64), th):
            t0 = max(tk - 2 * sigma, 0.0)  # ends before the hit: f keeps its sign on it
            cls, lo, hi, y0, rad = oracle.range_bound(mlp, p + (t0 + sigma / 2) * r, ((sigma / 2) * r)[None, :],
                                                      "fixed")
            assert cls == oracle.UNKNOWN and rad > abs(y0)
