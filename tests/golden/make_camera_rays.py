"""Writes camera_rays_elu512x6_pe.json: CastRay (Proc. 2; App. B step rule)
of the FP64 oracle for 64 pixels of the 1920x1080 pinhole camera at (0,0,3)
(looking at the origin, up +y, vertical field of view 40 degrees) against the
ELU 39(PE, 6 octaves)-[512]x6-1 network (He init, seed 2), affine-fixed,
delta 1e-4, t_max 10, sigma0 1, eta 1.5 / 0.5, safety 0.98, every ray marched
to its end or to 40,000 iterations. The pixels form an 8 x 8 grid of stride
64 centred on the image centre.

Calls only the oracle and the seeded input generators. Run from the
repository root: python tests/golden/make_camera_rays.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2202_02444_gb300 import workloads as wl  # noqa: E402

W, H = 1920, 1080
CAP = 40000
RAY = dict(delta=1e-4, t_max=10.0, sigma0=1.0, eta_plus=1.5, eta_minus=0.5, safety=0.98)


def pixels():
    return [(H // 2 - 224 + 64 * j) * W + (W // 2 - 224 + 64 * i) for j in range(8) for i in range(8)]


def main():
    mlp = wl.net_elu512x6_pe()
    o, d = wl.camera_rays(W, H)
    sel = pixels()
    t0 = time.time()
    r = oracle.cast_rays(mlp, o[sel], d[sel], "fixed", max_iters=CAP, **RAY)
    dt = time.time() - t0
    out = {"source": "FP64 oracle CastRay (Proc. 2, App. B), tests/golden/make_camera_rays.py",
           "network": "ELU 39(PE 6 octaves)-[512]x6-1, He init, seed 2",
           "camera": {"width": W, "height": H, "eye": [0, 0, 3], "vfov_deg": 40},
           "arith": "fixed", **RAY, "max_iters": CAP, "pixels": sel,
           "t": [float(x) if x == x and abs(x) != float("inf") else str(x) for x in r["t"]],
           "iters": [int(x) for x in r["iters"]], "status": [int(x) for x in r["status"]],
           "margin": [float(x) for x in r["margin"]],
           "oracle_seconds": round(dt, 1), "threads": oracle.max_threads()}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "camera_rays_elu512x6_pe.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, dt)


if __name__ == "__main__":
    main()
