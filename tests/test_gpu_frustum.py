"""Frustum ray casting (sra_cast_frustum, Sec. 4.3): every pixel's result
agrees with its own CastRay (Proc. 2) within the delta semantics, against
the FP32 ray kernel, the FP64 oracle and an analytic plane."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2202_02444_gb300 import workloads as wl

from test_gpu_rays import check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sra():
    from paper_2202_02444_gb300 import sra as s
    return s


def agree(a, b, delta):
    fa, fb = np.isfinite(a), np.isfinite(b)
    same = (fa == fb) & (np.isnan(a) == np.isnan(b))
    both = fa & fb
    same[both] &= np.abs(a[both] - b[both]) <= delta * 1.0001 + 1e-6
    return same


def test_frustum_matches_per_ray(sra):
    mlp = wl.net_small_relu()
    W, H = 96, 64
    o, d = wl.camera_rays(W, H)
    net = sra.Net(mlp)
    try:
        kw = dict(arith="fixed", delta=1e-3, max_iters=20000)
        t_f, it_f, stats = sra.cast_frustum(net, o[0], torch.from_numpy(d).cuda(), W, H, grid=8, **kw)
        t_r, it_r = sra.cast_rays(net, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), **kw)
        torch.cuda.synchronize()
        t_f, t_r = t_f.cpu().numpy(), t_r.cpu().numpy()
    finally:
        net.close()
    assert np.isfinite(t_r).sum() > 500  # the surface is in view
    assert agree(t_f, t_r, 1e-3).mean() >= 0.98
    # amortisation: frustum boxes + per-pixel iterations after the hand-over
    # cost less than marching every pixel from the eye
    assert stats["frustum_boxes"] + it_f.sum().item() < it_r.sum().item()
    # the oracle's CastRay on a sample of pixels
    idx = wl.sample_rows(W * H, 200, seed=1)
    ref = oracle.cast_rays(mlp, o[idx], d[idx], "fixed", delta=1e-3, max_iters=20000)
    check(t_f[idx], ref, 1e-3, 1e-4, max_frac=0.03)


def test_frustum_plane_analytic(sra):
    nv = np.array([0.3, -0.5, 0.8])
    mlp = wl.make_custom_mlp([3, 1], [], [(nv[None, :], np.array([-0.1]))])
    W, H = 40, 30
    o, d = wl.camera_rays(W, H)
    net = sra.Net(mlp)
    try:
        t, _, _ = sra.cast_frustum(net, o[0], torch.from_numpy(d).cuda(), W, H, grid=4, delta=1e-3)
        t = t.cpu().numpy()
    finally:
        net.close()
    n32 = nv.astype(np.float32).astype(np.float64)
    tstar = -(o.astype(np.float64) @ n32 + float(np.float32(-0.1))) / (d.astype(np.float64) @ n32)
    for i in range(W * H):
        if 1e-3 < tstar[i] < 10 - 1e-2:
            assert t[i] < tstar[i] + 1e-5 and tstar[i] <= t[i] + 1e-3 + 1e-5
        elif tstar[i] < 0 or tstar[i] > 10.1:
            assert math.isinf(t[i])


def test_frustum_bf16_handover(sra):
    mlp = wl.make_mlp([128] * 3, "elu", seed=51, pe_octaves=2)
    W, H = 64, 48
    o, d = wl.camera_rays(W, H)
    net = sra.Net(mlp)
    try:
        kw = dict(arith="fixed", delta=1e-3, max_iters=6000)
        t_b, _, st = sra.cast_frustum(net, o[0], torch.from_numpy(d).cuda(), W, H, precision="bf16", **kw)
        t_f, _, _ = sra.cast_frustum(net, o[0], torch.from_numpy(d).cuda(), W, H, precision="fp32", **kw)
        torch.cuda.synchronize()
        sra.sync_status(net)
    finally:
        net.close()
    assert agree(t_b.cpu().numpy(), t_f.cpu().numpy(), 1e-3).mean() >= 0.97
    assert st["rays"] > 0
