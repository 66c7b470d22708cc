"""GPU parity of the tensor-core CastRay path (precision "bf16": split-BF16
hidden layers on tcgen05, FP32 elsewhere) against the FP64 oracle and
against the FP32 SIMT ray kernel (Proc. 2)."""
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


def cast(sra, mlp, o, d, **kw):
    net = sra.Net(mlp)
    try:
        t, it = sra.cast_rays(net, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), **kw)
        torch.cuda.synchronize()
        sra.sync_status(net)
    finally:
        net.close()
    return t.cpu().numpy(), it.cpu().numpy()


@pytest.mark.parametrize("width,depth,act,pe", [
    (128, 3, "relu", 0),
    (128, 4, "elu", 3),
    (128, 3, "sin", 0),
    (256, 3, "relu", 2),
])
def test_tc_rays_vs_oracle(sra, width, depth, act, pe):
    mlp = wl.make_mlp([width] * depth, act, seed=31 + width + depth, pe_octaves=pe)
    o, d = wl.sphere_rays(203, seed=8, radius=2.0)  # ragged against 8 slots per CTA
    t, it = cast(sra, mlp, o, d, arith="fixed", precision="bf16", delta=1e-3, max_iters=4000)
    ref = oracle.cast_rays(mlp, o, d, "fixed", delta=1e-3, max_iters=4000)
    check(t, ref, 1e-3, 1e-3, max_frac=0.05)
    assert np.isfinite(t).sum() + np.isinf(t).sum() > 150


def test_tc_rays_relu256x8(sra):
    """The 3-[256]x8-1 ReLU net: seven hidden layers on the tensor cores."""
    mlp = wl.net_relu256x8()
    o, d = wl.sphere_rays(96, seed=9, radius=2.0)
    t, it = cast(sra, mlp, o, d, arith="fixed", precision="bf16", delta=1e-3, max_iters=3000)
    ref = oracle.cast_rays(mlp, o, d, "fixed", delta=1e-3, max_iters=3000)
    check(t, ref, 1e-3, 1e-3, max_frac=0.05)


def test_tc_rays_camera_elu512_pe_sample(sra):
    """39(PE)-[512]x6-1 ELU net, sampled pixels of the 1920x1080 camera at
    (0,0,3), delta 1e-4, both sides capped at 300 iterations."""
    mlp = wl.net_elu512x6_pe()
    o, d = wl.camera_rays(1920, 1080)
    idx = wl.sample_rows(len(o), 8, seed=4)
    t, it = cast(sra, mlp, o[idx], d[idx], arith="fixed", precision="bf16", delta=1e-4, max_iters=300)
    ref = oracle.cast_rays(mlp, o[idx], d[idx], "fixed", delta=1e-4, max_iters=300)
    check(t, ref, 1e-4, 1e-3, max_frac=0.25)


def test_tc_rays_match_fp32_kernel(sra):
    """Many rays, no oracle: the tensor-core and the FP32 SIMT kernels agree on
    hit / miss and on t within delta for nearly every ray."""
    mlp = wl.make_mlp([128] * 4, "elu", seed=40, pe_octaves=2)
    o, d = wl.sphere_rays(2000, seed=10, radius=2.0)
    kw = dict(arith="fixed", delta=1e-3, max_iters=6000)
    t_tc, it_tc = cast(sra, mlp, o, d, precision="bf16", **kw)
    t_32, it_32 = cast(sra, mlp, o, d, precision="fp32", **kw)
    hit_tc, hit_32 = np.isfinite(t_tc), np.isfinite(t_32)
    same = (hit_tc == hit_32) & (np.isnan(t_tc) == np.isnan(t_32))
    both = hit_tc & hit_32
    same[both] &= np.abs(t_tc[both] - t_32[both]) <= 1e-3 * 1.0001 + 1e-6
    assert same.mean() >= 0.97, same.mean()
    assert hit_tc.sum() > 200


def test_tc_rays_iteration_cap(sra):
    mlp = wl.make_mlp([128] * 3, "relu", seed=41)
    o, d = wl.sphere_rays(40, seed=5, radius=2.0)
    t, it = cast(sra, mlp, o, d, arith="fixed", precision="bf16", delta=1e-3, max_iters=2)
    assert np.all(it <= 2) and np.all(it >= 1)
    assert np.isnan(t).any()


def test_tc_rays_unsupported(sra):
    o, d = wl.sphere_rays(8, seed=5, radius=2.0)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    cases = [(wl.make_mlp([128, 64, 128], "relu", seed=1), "fixed"),  # non-uniform width
             (wl.make_mlp([96] * 3, "relu", seed=1), "fixed"),        # width not 128/256/512
             (wl.make_mlp([128] * 3, "relu", seed=1), "truncate")]    # not affine-fixed
    for mlp, arith in cases:
        net = sra.Net(mlp)
        try:
            with pytest.raises(sra.SraError) as e:
                sra.cast_rays(net, ot, dt, arith=arith, K=4, precision="bf16")
            assert e.value.code == sra.EUNSUPPORTED
        finally:
            net.close()
