"""GPU parity of the tensor-core CastRay path (precision "bf16": split-BF16
hidden layers on tcgen05, FP32 elsewhere; "bf16_sound": the same with an
a-priori rounding radius on every segment bound) against the FP64 oracle,
an analytic plane, and the FP32 SIMT ray kernel (Proc. 2)."""
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


def cast(sra, mlp, o, d, **kw):
    net = sra.Net(mlp)
    try:
        t, it = sra.cast_rays(net, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), **kw)
        torch.cuda.synchronize()
        sra.sync_status(net)
    finally:
        net.close()
    return t.cpu().numpy(), it.cpu().numpy()


@pytest.mark.parametrize("precision", ["bf16", "bf16_sound"])
@pytest.mark.parametrize("width,depth,act,pe", [
    (128, 3, "relu", 0),
    (128, 4, "elu", 3),
    (128, 3, "sin", 0),
    (256, 3, "relu", 2),
    (512, 3, "elu", 2),
])
def test_tc_rays_vs_oracle(sra, width, depth, act, pe, precision):
    """Hit / miss and t within delta against the oracle's CastRay. The sound
    form's segment bounds carry the a-priori rounding radius, so they decide
    fewer segments and the march takes more steps: it runs without an
    effective cap (t_max / delta + 2000 iterations)."""
    mlp = wl.make_mlp([width] * depth, act, seed=31 + width + depth, pe_octaves=pe)
    o, d = wl.sphere_rays(203, seed=8, radius=2.0)  # ragged against 8 slots per CTA
    cap = 4000 if precision == "bf16" else 12000
    t, it = cast(sra, mlp, o, d, arith="fixed", precision=precision, delta=1e-3, max_iters=cap)
    ref = oracle.cast_rays(mlp, o, d, "fixed", delta=1e-3, max_iters=cap)
    check(t, ref, 1e-3, 1e-3, max_frac=0.05)
    assert np.isfinite(t).sum() + np.isinf(t).sum() > 150


def plane_net(width, nv, b, M=16.0):
    """f(x) = nv . x + b through two ReLU layers of the given width: neuron 0
    carries nv . x + b + M (positive on every ray's path, so both ReLUs act
    as the identity there) and the output subtracts M; the other neurons are
    zero."""
    W0 = np.zeros((width, 3))
    W0[0] = nv
    b0 = np.zeros(width)
    b0[0] = b + M
    W1 = np.zeros((width, width))
    W1[0, 0] = 1.0
    W2 = np.zeros((1, width))
    W2[0, 0] = 1.0
    return wl.make_custom_mlp([3, width, width, 1], [wl.ACT_RELU, wl.ACT_RELU],
                              [(W0, b0), (W1, np.zeros(width)), (W2, np.array([-M]))])


@pytest.mark.parametrize("precision", ["bf16", "bf16_sound"])
@pytest.mark.parametrize("width", [128, 512])
def test_tc_rays_plane_analytic(sra, width, precision):
    """A plane through the tensor-core path: segment bounds of a linear
    function decide their sign (up to the rounding radius), so the march
    takes long steps, and every hit lies within delta after the analytic
    crossing t*, none before it (Sec. 4.1's delta semantics), up to the
    precision of the point test: f at t + delta is evaluated with BF16 hi/lo
    operands (16 significant bits, here about 1e-4 in t at |x| ~ 10). A
    sound segment bound that wrongly decided a segment holding the crossing
    would step over it by more than that."""
    nv = np.array([0.3, -0.5, 0.8])
    mlp = plane_net(width, nv, -0.1)
    o, d = wl.sphere_rays(300, seed=3)
    t, it = cast(sra, mlp, o, d, arith="fixed", precision=precision, delta=1e-3, max_iters=20000)
    n32 = nv.astype(np.float32).astype(np.float64)
    tstar = -(o.astype(np.float64) @ n32 + float(np.float32(-0.1))) / (d.astype(np.float64) @ n32)
    hits = 0
    for i in range(len(o)):
        if 1e-3 < tstar[i] < 10 - 1e-2:
            assert t[i] < tstar[i] + 2e-4 and tstar[i] <= t[i] + 1e-3 + 2e-4, (i, t[i], tstar[i])
            hits += 1
        elif tstar[i] < 0 or tstar[i] > 10.1:
            assert math.isinf(t[i]), (i, t[i], tstar[i])
    assert hits > 50
    # long steps: far fewer iterations than t / delta
    assert np.median(it) < 100, np.median(it)


def zero_padded(mlp, H):
    """The same network written out with every hidden layer H wide (zero
    weights, biases and output weights in the padding)."""
    layers = []
    for l in range(mlp.n_layers):
        W, b = mlp.layer(l)
        o = H if l + 1 < mlp.n_layers else 1
        i = mlp.widths[0] if l == 0 else H
        Wp = np.zeros((o, i), np.float32)
        bp = np.zeros(o, np.float32)
        Wp[:W.shape[0], :W.shape[1]] = W
        bp[:b.shape[0]] = b
        layers.append((Wp, bp))
    return wl.make_custom_mlp([mlp.widths[0]] + [H] * (mlp.n_layers - 1) + [1], mlp.acts, layers,
                              pe_octaves=mlp.pe_octaves)


@pytest.mark.parametrize("precision", ["bf16", "bf16_sound"])
@pytest.mark.parametrize("hidden,act,pe,H", [([64] * 3, "relu", 0, 128), ([96, 200, 128], "elu", 2, 256),
                                             ([40, 40, 40, 40], "sin", 0, 128)])
def test_tc_rays_padded_widths(sra, hidden, act, pe, H, precision):
    """Hidden layers narrower than the kernel's width (128, 256 or 512) run on
    weights padded with zeros: every ray's t and iteration count equal, bit
    for bit, those of the same network written out at that width, and
    against the oracle the usual CastRay gate holds."""
    mlp = wl.make_mlp(hidden, act, seed=70 + len(hidden), pe_octaves=pe)
    o, d = wl.sphere_rays(203, seed=9, radius=2.0)
    kw = dict(arith="fixed", precision=precision, delta=1e-3, max_iters=4000 if precision == "bf16" else 12000)
    t, it = cast(sra, mlp, o, d, **kw)
    t2, it2 = cast(sra, zero_padded(mlp, H), o, d, **kw)
    assert np.array_equal(t, t2, equal_nan=True) and np.array_equal(it, it2)
    ref = oracle.cast_rays(mlp, o, d, "fixed", delta=1e-3, max_iters=kw["max_iters"])
    check(t, ref, 1e-3, 1e-3, max_frac=0.05)


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
    cases = [(wl.make_mlp([128] * 10, "relu", seed=1), "fixed", "bf16", "chebyshev"),     # 9 hidden H -> H layers
             (wl.make_mlp([128] * 3, "relu", seed=1, pe_octaves=11), "fixed", "bf16", "chebyshev"),  # 69 inputs
             (wl.make_mlp([128] * 3, "relu", seed=1), "truncate", "bf16", "chebyshev"),   # not affine-fixed
             (wl.make_mlp([128] * 3, "relu", seed=1), "fixed", "bf16_sound", "minrange")]  # sound: Chebyshev only
    for mlp, arith, prec, slope in cases:
        net = sra.Net(mlp)
        try:
            with pytest.raises(sra.SraError) as e:
                sra.cast_rays(net, ot, dt, arith=arith, K=4, precision=prec, slope=slope)
            assert e.value.code == sra.EUNSUPPORTED
        finally:
            net.close()
