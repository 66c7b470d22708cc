"""CastRay (Proc. 2) in FP64 on the GPU and the FP64 re-check of rays that
met a near-zero decision (the FP32 SIMT and the BF16 tensor-core march).

The re-check marches a flagged ray again from its start in FP64, so with a
band wide enough to flag every ray the results must be those of the FP64
march bit for bit, and with any band every ray carries either its own
lower-precision result or its FP64 result."""
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


def cast(sra, net, o, d, **kw):
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    opts = sra.make_opts(recheck_count=count, **kw)
    t, it = sra.cast_rays(net, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), opts=opts)
    torch.cuda.synchronize()
    sra.sync_status(net)
    return t.cpu().numpy(), it.cpu().numpy(), int(count.item())


def same(a, b):
    """Bitwise equality of float arrays (NaN and inf included)."""
    return np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("arith,K", [("fixed", 0), ("truncate", 8)])
def test_fp64_rays_vs_oracle(sra, arith, K):
    mlp = wl.net_small_relu()
    o, d = wl.sphere_rays(300, seed=5, radius=2.0)
    net = sra.Net(mlp)
    try:
        t, it, cnt = cast(sra, net, o, d, arith=arith, K=K, delta=1e-3, precision="fp64")
    finally:
        net.close()
    assert cnt == 0  # no re-check in FP64
    ref = oracle.cast_rays(mlp, o, d, arith, K=K, delta=1e-3)
    # both march in FP64: only near-ties of the order of FP64 rounding may differ
    check(t, ref, 1e-3, 1e-9, max_frac=0.01)
    assert np.isfinite(t).sum() > 50


@pytest.mark.parametrize("prec,mlp_fn", [
    ("fp32", lambda: wl.net_small_relu()),
    ("fp32", lambda: wl.make_mlp([64, 64], "elu", seed=24, pe_octaves=3)),
    ("bf16", lambda: wl.make_mlp([128] * 4, "elu", seed=35, pe_octaves=3)),
])
def test_recheck_every_ray_equals_fp64(sra, prec, mlp_fn):
    """A band that flags every step: every ray is marched again in FP64."""
    mlp = mlp_fn()
    o, d = wl.sphere_rays(203, seed=8, radius=2.0)
    net = sra.Net(mlp)
    try:
        kw = dict(arith="fixed", delta=1e-3, max_iters=4000)
        t64, it64, c64 = cast(sra, net, o, d, precision="fp64", **kw)
        t, it, cnt = cast(sra, net, o, d, precision=prec, recheck=True, recheck_band=1e30, **kw)
    finally:
        net.close()
    assert c64 == 0
    assert cnt == len(o)
    assert same(t, t64) and np.array_equal(it, it64)


@pytest.mark.parametrize("prec,band", [("fp32", 1e-5), ("fp32", 3e-2), ("bf16", 1e-5), ("bf16", 3e-2)])
def test_recheck_keeps_own_or_fp64_result(sra, prec, band):
    """Every ray ends with its own result or its FP64 result; every ray whose
    result changed was counted; a wide band flags some rays."""
    mlp = wl.make_mlp([128] * 3, "elu", seed=41, pe_octaves=2)
    o, d = wl.sphere_rays(256, seed=9, radius=2.0)
    net = sra.Net(mlp)
    try:
        kw = dict(arith="fixed", delta=1e-3, max_iters=4000)
        t0, it0, c0 = cast(sra, net, o, d, precision=prec, **kw)
        t64, it64, _ = cast(sra, net, o, d, precision="fp64", **kw)
        t, it, cnt = cast(sra, net, o, d, precision=prec, recheck=True, recheck_band=band, **kw)
    finally:
        net.close()
    assert c0 == 0
    as_own = (t.view(np.uint32) == t0.view(np.uint32)) & (it == it0)
    as_64 = (t.view(np.uint32) == t64.view(np.uint32)) & (it == it64)
    assert np.all(as_own | as_64)
    changed = int((~as_own).sum())
    assert changed <= cnt <= len(o)
    if band > 1e-3:
        assert cnt > 0


def test_recheck_count_of_boxes(sra):
    """sra_bound_boxes counts the boxes its FP64 re-check took again."""
    mlp = wl.net_small_relu()
    c, h = wl.make_boxes(1000, seed=3, hw_lo=1 / 256, hw_hi=1 / 4)
    net = sra.Net(mlp)
    try:
        C_, H_ = torch.from_numpy(c).cuda(), torch.from_numpy(h).cuda()
        counts = []
        for band in (0.0, 1e-2, 1e30):
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            o = sra.make_opts(arith="fixed", recheck=True, recheck_band=band, recheck_count=cnt)
            lo, hi, _ = sra.bound_boxes(net, C_, H_, opts=o)
            torch.cuda.synchronize()
            counts.append(int(cnt.item()))
            if band == 1e-2:  # the boxes within the band, judged on the FP32 bound
                o32 = sra.make_opts(arith="fixed")
                lo32, hi32, _ = sra.bound_boxes(net, C_, H_, opts=o32)
                l, u = lo32.cpu().numpy().astype(np.float64), hi32.cpu().numpy().astype(np.float64)
                y0, rad = (l + u) / 2, (u - l) / 2
                near = (np.abs(l) <= band * (np.abs(y0) + rad)) | (np.abs(u) <= band * (np.abs(y0) + rad))
                assert abs(counts[-1] - int(near.sum())) <= max(2, int(0.01 * len(near)))
    finally:
        net.close()
    assert counts[0] <= counts[1] <= counts[2] == 1000
