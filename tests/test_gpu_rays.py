"""GPU parity of sra_cast_rays (Proc. 2) against the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2202_02444_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sra():
    from paper_2202_02444_gb300 import sra as s
    return s


def cast(sra, mlp, o, d, **kw):
    net = sra.Net(mlp)
    t, it = sra.cast_rays(net, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), **kw)
    torch.cuda.synchronize()
    net.close()
    return t.cpu().numpy(), it.cpu().numpy()


def check(t, ref, delta, margin_band, max_frac=0.02):
    """Hit/miss agree and |t - t_ref| <= delta. The adaptive step keeps its
    segment bounds close to zero by design, so FP32 and FP64 trajectories
    may differ; both answers are then correct to the delta semantics of
    Sec. 4.1 and still agree within delta. A ray may differ only if the
    oracle's trajectory met a value or bound within margin_band of zero, and
    at most max_frac of the rays may."""
    hit_g, hit_r = np.isfinite(t), ref["status"] == 1
    cap_g, cap_r = np.isnan(t), ref["status"] == 2
    with np.errstate(invalid="ignore"):  # inf - inf on misses, masked out below
        far = hit_g & hit_r & (np.abs(t - ref["t"]) > delta * 1.0001 + 1e-6)
    mism = (hit_g != hit_r) | (cap_g != cap_r) | far
    unexplained = mism & (ref["margin"] >= margin_band)
    assert not unexplained.any(), np.nonzero(unexplained)[0][:10]
    assert mism.sum() <= max_frac * len(t) + 1, int(mism.sum())
    return int(mism.sum())


@pytest.mark.parametrize("arith,K", [("fixed", 0), ("truncate", 8), ("interval", 0)])
def test_small_relu_rays(sra, arith, K):
    mlp = wl.net_small_relu()
    o, d = wl.sphere_rays(300, seed=5, radius=2.0)  # ragged against the slot count
    t, it = cast(sra, mlp, o, d, arith=arith, K=K, delta=1e-3)
    ref = oracle.cast_rays(mlp, o, d, arith, K=K, delta=1e-3)
    check(t, ref, 1e-3, 1e-4)
    assert (np.isfinite(t)).sum() > 50


def test_elu_pe_rays(sra):
    mlp = wl.make_mlp([64, 64], "elu", seed=24, pe_octaves=3)
    o, d = wl.sphere_rays(64, seed=6, radius=2.0)
    t, it = cast(sra, mlp, o, d, arith="fixed", delta=1e-3)
    ref = oracle.cast_rays(mlp, o, d, "fixed", delta=1e-3)
    check(t, ref, 1e-3, 1e-4, max_frac=0.05)


def test_plane_rays_analytic(sra):
    nv = np.array([0.3, -0.5, 0.8])
    mlp = wl.make_custom_mlp([3, 1], [], [(nv[None, :], np.array([-0.1]))])
    o, d = wl.sphere_rays(200, seed=3)
    t, _ = cast(sra, mlp, o, d, delta=1e-3)
    n32 = nv.astype(np.float32).astype(np.float64)
    tstar = -(o.astype(np.float64) @ n32 + float(np.float32(-0.1))) / (d.astype(np.float64) @ n32)
    for i in range(200):
        if 1e-3 < tstar[i] < 10 - 1e-2:
            assert t[i] < tstar[i] + 1e-5 and tstar[i] <= t[i] + 1e-3 + 1e-5
        elif tstar[i] < 0 or tstar[i] > 10.1:
            assert math.isinf(t[i])


def test_iteration_cap_reports_nan(sra):
    mlp = wl.net_small_relu()
    o, d = wl.sphere_rays(40, seed=5, radius=2.0)
    t, it = cast(sra, mlp, o, d, delta=1e-3, max_iters=2)
    assert np.all(it <= 2)
    assert np.all(np.isnan(t) | np.isfinite(t))
    assert np.isnan(t).any()


def test_camera_rays_elu512_pe_sample(sra):
    """The 39(PE)-[512]x6-1 ELU net with a 1920x1080 camera at (0,0,3):
    sampled pixel rays against the oracle (delta = 1e-4)."""
    mlp = wl.net_elu512x6_pe()
    o, d = wl.camera_rays(1920, 1080)
    idx = wl.sample_rows(len(o), 8, seed=4)
    # both sides stop at the same iteration cap (the oracle costs ~10 ms per
    # iteration of this net); capped rays must be capped on both sides
    t, it = cast(sra, mlp, o[idx], d[idx], arith="fixed", delta=1e-4, max_iters=300)
    ref = oracle.cast_rays(mlp, o[idx], d[idx], "fixed", delta=1e-4, max_iters=300)
    check(t, ref, 1e-4, 1e-5, max_frac=0.25)
