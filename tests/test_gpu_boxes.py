"""GPU parity of sra_bound_boxes (Proc. 1) against the FP64 oracle, through
the C ABI, on seeded boxes; plus soundness against dense samples."""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_02444_gb300 import workloads as wl
from tests.np_forward import box_samples, forward
from tests.parity import FP32_REL, FP64_REL, assert_parity, compare_bounds, soundness_violations

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sra():
    from paper_2202_02444_gb300 import sra as s
    return s


def run(sra, mlp, c, h, **kw):
    net = sra.Net(mlp)
    lo, hi, cls = sra.bound_boxes(net, torch.from_numpy(c).cuda(), torch.from_numpy(h).cuda(), **kw)
    torch.cuda.synchronize()
    out = lo.cpu().numpy(), hi.cpu().numpy(), cls.cpu().numpy()
    net.close()
    return out


CASES = [("fixed", 0), ("truncate", 8), ("full", 0), ("interval", 0)]


@pytest.mark.parametrize("arith,K", CASES)
@pytest.mark.parametrize("slope", ["chebyshev", "minrange"])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_small_relu_4096_boxes(sra, arith, K, slope, precision):
    """ReLU 3-32-32-1 on the 4096 standalone boxes (log-uniform half-widths)."""
    mlp = wl.net_small_relu()
    c, h = wl.make_boxes(4096, seed=100)
    lo, hi, cls = run(sra, mlp, c, h, arith=arith, K=K, slope=slope, precision=precision)
    ref = oracle.bound_boxes(mlp, c, h, arith, K=K, slope=slope)
    rel = FP32_REL if precision == "fp32" else FP64_REL
    rep = compare_bounds(lo, hi, cls, ref, rel=rel, zero_band=1e-6)
    assert_parity(rep)


NETS = {
    "elu": lambda: wl.make_mlp([48, 48, 48], "elu", seed=22),
    "sin": lambda: wl.make_mlp([40, 40], "sin", seed=23),
    "elu_pe": lambda: wl.make_mlp([64, 64], "elu", seed=24, pe_octaves=3),
    "relu_deep": lambda: wl.make_mlp([96] * 5, "relu", seed=25),
}


@pytest.mark.parametrize("name", list(NETS))
@pytest.mark.parametrize("arith,K", [("fixed", 0), ("truncate", 16), ("interval", 0)])
def test_activation_families(sra, name, arith, K):
    mlp = NETS[name]()
    hw = 0.25 if name in ("elu", "relu_deep") else 0.03
    c, h = wl.make_boxes(700, seed=3, hw_hi=hw)  # 700: ragged against any boxes-per-CTA
    lo, hi, cls = run(sra, mlp, c, h, arith=arith, K=K)
    ref = oracle.bound_boxes(mlp, c, h, arith, K=K)
    assert_parity(compare_bounds(lo, hi, cls, ref))
    lo64, hi64, cls64 = run(sra, mlp, c, h, arith=arith, K=K, precision="fp64")
    assert_parity(compare_bounds(lo64, hi64, cls64, ref, rel=FP64_REL))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_relu256x8_truncate64_sample(sra, precision):
    """The 3-[256]x8-1 ReLU net, affine-truncate K=64, on sampled boxes of
    the sizes its depth-10 octree visits."""
    mlp = wl.net_relu256x8()
    rng = np.random.default_rng(5)
    lev = rng.integers(2, 11, 96)
    c = rng.uniform(-1, 1, (96, 3)).astype(np.float32)
    h = np.repeat((1.0 / (1 << lev))[:, None], 3, 1).astype(np.float32)
    lo, hi, cls = run(sra, mlp, c, h, arith="truncate", K=64, precision=precision)
    ref = oracle.bound_boxes(mlp, c, h, "truncate", K=64)
    rel = FP32_REL if precision == "fp32" else FP64_REL
    assert_parity(compare_bounds(lo, hi, cls, ref, rel=rel), max_tie_frac=0.1)


@pytest.mark.parametrize("hw_lo,hw_hi", [(1e-5, 1e-3), (1e-3, 1e-2)])
def test_elu512x6_pe_fixed_sample(sra, hw_lo, hw_hi):
    """The 39(PE)-[512]x6-1 ELU net, affine-fixed, on segment-sized and larger
    boxes (the bound grows to radii of 1e3..1e7 through the six 512-wide
    layers). FP32 is held to the 1e-5 gate on both: a float32 emulation of
    the same bound drifts from FP64 by less than 1e-6 there
    (tests/test_fp32_drift.py). The FP64 path is held to 1e-9."""
    mlp = wl.net_elu512x6_pe()
    c, h = wl.make_boxes(24, seed=12, hw_lo=hw_lo, hw_hi=hw_hi)
    ref = oracle.bound_boxes(mlp, c, h, "fixed")
    lo, hi, cls = run(sra, mlp, c, h, arith="fixed")
    assert_parity(compare_bounds(lo, hi, cls, ref, rel=FP32_REL))
    lo, hi, cls = run(sra, mlp, c, h, arith="fixed", precision="fp64")
    assert_parity(compare_bounds(lo, hi, cls, ref, rel=FP64_REL))


@pytest.mark.parametrize("arith,K", [("fixed", 0), ("truncate", 8), ("interval", 0)])
def test_soundness_dense_samples(sra, arith, K):
    """Sampled f (independent numpy FP64 forward pass) lies in the FP32 bound
    within FP32 rounding (the fuzz test of Sec. 3.6)."""
    mlp = wl.net_small_relu()
    c, h = wl.make_boxes(256, seed=77)
    lo, hi, _ = run(sra, mlp, c, h, arith=arith, K=K)
    f = np.stack([forward(mlp, box_samples(c[i], h[i], seed=i)) for i in range(256)])
    assert soundness_violations(lo, hi, f, tol_rel=1e-5) == 0


def test_edge_sizes(sra):
    mlp = wl.net_small_relu()
    net = sra.Net(mlp)
    z = torch.empty((0, 3), dtype=torch.float32, device="cuda")
    lo, hi, cls = sra.bound_boxes(net, z, z)
    assert lo.numel() == 0
    c, h = wl.make_boxes(1, seed=1)
    lo, hi, cls = sra.bound_boxes(net, torch.from_numpy(c).cuda(), torch.from_numpy(h).cuda())
    ref = oracle.bound_boxes(mlp, c, h)
    assert_parity(compare_bounds(lo.cpu().numpy(), hi.cpu().numpy(), cls.cpu().numpy(), ref))
    net.close()


def test_zero_width_boxes_equal_point_values(sra):
    """A degenerate box (all half-widths 0) bounds exactly f(center)."""
    mlp = NETS["elu_pe"]()
    c, _ = wl.make_boxes(333, seed=4)
    h = np.zeros_like(c)
    lo, hi, cls = run(sra, mlp, c, h, arith="interval")
    f = forward(mlp, c)
    np.testing.assert_allclose(lo, f, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(hi, f, rtol=1e-5, atol=1e-5)


def test_large_batch_sampled(sra):
    """2^20 boxes in one call (ragged grid tail), sampled oracle parity and
    class / range consistency on every box."""
    mlp = wl.net_small_relu()
    n = (1 << 20) + 37
    c, h = wl.make_boxes(n, seed=101)
    lo, hi, cls = run(sra, mlp, c, h, arith="fixed")
    assert np.all(hi >= lo)
    k = np.where(lo > 0, 1, np.where(hi < 0, 2, 0))
    assert np.array_equal(k, cls)
    idx = wl.sample_rows(n, 3000, seed=2)
    idx = np.concatenate([idx, [n - 1]])
    ref = oracle.bound_boxes(mlp, c[idx], h[idx], "fixed")
    assert_parity(compare_bounds(lo[idx], hi[idx], cls[idx], ref))


def test_recheck_makes_classes_exact(sra):
    """With the FP64 re-check, UNKNOWN boxes near zero take the FP64 class:
    classes then equal the oracle's except at exact FP64 ties."""
    mlp = wl.net_small_relu()
    c, h = wl.make_boxes(4096, seed=100)
    lo, hi, cls = run(sra, mlp, c, h, arith="fixed", recheck=True, recheck_band=1e-4)
    ref = oracle.bound_boxes(mlp, c, h, "fixed")
    near = np.minimum(np.abs(ref["lo"]), np.abs(ref["hi"])) <= 1e-12 * (1 + np.abs(ref["y0"]) + ref["rad"])
    assert np.all((cls == ref["cls"]) | near)


def test_eval_matches_numpy(sra):
    for name in ("elu_pe", "sin", "relu_deep"):
        mlp = NETS[name]()
        x = np.random.default_rng(1).uniform(-1, 1, (1001, 3)).astype(np.float32)
        net = sra.Net(mlp)
        y = sra.evaluate(net, torch.from_numpy(x).cuda()).cpu().numpy()
        net.close()
        np.testing.assert_allclose(y, forward(mlp, x), rtol=1e-4, atol=1e-5)
