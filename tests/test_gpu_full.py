"""GPU parity of affine-full RangeBound past 128 noise symbols (Sec. 3.3
"full" keeps every symbol) against the FP64 oracle, through the C ABI.

The paper's experiments use 8-layer, 32-wide networks (seven ReLU / ELU
hidden layers): affine-full reaches 3 + 7 * 32 = 227 symbols there, which
the shared-memory full kernel serves (the SIMT engine's register row holds
128). Wider networks, and networks with the positional encoding, keep each
box's noise matrix in device memory (3-[256]x8-1: 2051 symbols, 2.1 MB per
box) and run every dense layer as one batched GEMM over the boxes of a pass.
Checks: boxes in FP32 and FP64 for ReLU / ELU / sin networks of width 32-256
with and without the encoding, ragged counts, several passes, an octree round
with FP64 re-check, and soundness against dense samples.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_02444_gb300 import workloads as wl
from tests.np_forward import box_samples, forward
from tests.parity import FP32_REL, FP64_REL, assert_parity, compare_bounds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sra():
    from paper_2202_02444_gb300 import sra as s
    return s


NETS = {
    # name: (network, half-width bound of the boxes)
    "relu32x7": (lambda: wl.make_mlp([32] * 7, "relu", seed=41), 0.25),   # 227 symbols
    "elu48x4": (lambda: wl.make_mlp([48] * 4, "elu", seed=42), 0.25),     # 195
    "sin40x4": (lambda: wl.make_mlp([40] * 4, "sin", seed=43), 0.02),     # 163
    "relu64x5": (lambda: wl.make_mlp([64] * 5, "relu", seed=44), 0.1),    # 323
}


def run_boxes(sra, mlp, c, h, **kw):
    net = sra.Net(mlp)
    lo, hi, cls = sra.bound_boxes(net, torch.from_numpy(c).cuda(), torch.from_numpy(h).cuda(), **kw)
    torch.cuda.synchronize()
    out = lo.cpu().numpy(), hi.cpu().numpy(), cls.cpu().numpy()
    net.close()
    return out


@pytest.mark.parametrize("name", list(NETS))
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_full_past_register_row(sra, name, precision):
    make, hw = NETS[name]
    mlp = make()
    c, h = wl.make_boxes(333, seed=7, hw_hi=hw)  # ragged against any grid
    lo, hi, cls = run_boxes(sra, mlp, c, h, arith="full", precision=precision)
    ref = oracle.bound_boxes(mlp, c, h, "full")
    rel = FP32_REL if precision == "fp32" else FP64_REL
    assert_parity(compare_bounds(lo, hi, cls, ref, rel=rel))


def test_full_tighter_than_truncate(sra):
    """Keeping every symbol never loses to truncation on the same boxes
    (aggregate, the ordering of Table 1's decided lengths)."""
    mlp = NETS["relu32x7"][0]()
    c, h = wl.make_boxes(512, seed=9, hw_hi=0.25)
    lo_f, hi_f, _ = run_boxes(sra, mlp, c, h, arith="full")
    lo_t, hi_t, _ = run_boxes(sra, mlp, c, h, arith="truncate", K=16)
    assert np.mean(hi_f - lo_f) < np.mean(hi_t - lo_t)


def test_full_contains_samples(sra):
    mlp = NETS["elu48x4"][0]()
    c, h = wl.make_boxes(64, seed=11, hw_hi=0.25)
    lo, hi, cls = run_boxes(sra, mlp, c, h, arith="full")
    for i in range(len(c)):
        f = forward(mlp, box_samples(c[i], h[i], n_grid=4, n_rand=128, seed=i))
        scale = abs(lo[i]) + abs(hi[i])
        assert f.min() >= lo[i] - 1e-5 * scale and f.max() <= hi[i] + 1e-5 * scale
        if cls[i] == 1:
            assert f.min() > 0
        if cls[i] == 2:
            assert f.max() < 0


def test_full_octree_round_with_recheck(sra):
    """One round of Proc. 3 with affine-full on the 32-wide net: classes
    match the oracle's on every node away from zero; children follow."""
    mlp = NETS["relu32x7"][0]()
    net = sra.Net(mlp)
    nodes = wl.random_nodes(1001, level=4, seed=13)
    fr = sra.nodes_to_tensor(nodes)
    out, leaves, counts = sra.classify_and_split(net, fr, 5, arith="full", recheck=True, recheck_band=1e-5)
    torch.cuda.synchronize()
    cnt = counts.cpu().numpy()
    cls_ref, lo_ref, hi_ref, _ = oracle.classify_nodes(mlp, nodes, (-1, -1, -1), (1, 1, 1), oracle.OCTREE,
                                                       "full")
    scale = 0.5 * (np.abs(lo_ref + hi_ref) + (hi_ref - lo_ref))
    near = np.minimum(np.abs(lo_ref), np.abs(hi_ref)) <= 1e-6 * (1.0 + scale)
    for code, slot in ((1, 2), (2, 3)):
        sure = int(np.sum((cls_ref == code) & ~near))
        assert sure <= cnt[slot] <= sure + int(near.sum()), (code, cnt, sure, int(near.sum()))
    assert cnt[2] + cnt[3] + cnt[4] == len(nodes)
    assert cnt[0] == 8 * cnt[4]
    net.close()


WIDE = {
    # name: (network, half-width bound of the boxes); symbols after the last layer
    "relu128x3": (lambda: wl.make_mlp([128] * 3, "relu", seed=61), 1 / 16),               # 387
    "elu128x3": (lambda: wl.make_mlp([128] * 3, "elu", seed=62), 1 / 16),                 # 387
    "sin128x3": (lambda: wl.make_mlp([128] * 3, "sin", seed=63), 1 / 256),                # 387
    "relu256x4": (lambda: wl.make_mlp([256] * 4, "relu", seed=64), 1 / 32),               # 1027
    "elu_pe2_128x3": (lambda: wl.make_mlp([128] * 3, "elu", seed=65, pe_octaves=2), 1 / 64),  # 399
    "elu_pe3_32x4": (lambda: wl.make_mlp([32] * 4, "elu", seed=45, pe_octaves=3), 1 / 64),    # 149
    "relu96x2": (lambda: wl.make_mlp([96] * 2, "relu", seed=46), 0.1),                    # 195
}


@pytest.mark.parametrize("name", list(WIDE))
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_full_in_device_memory(sra, name, precision):
    make, hw = WIDE[name]
    mlp = make()
    c, h = wl.make_boxes(97, seed=17, hw_lo=hw / 16, hw_hi=hw)
    lo, hi, cls = run_boxes(sra, mlp, c, h, arith="full", precision=precision)
    ref = oracle.bound_boxes(mlp, c, h, "full")
    rel = FP32_REL if precision == "fp32" else FP64_REL
    assert_parity(compare_bounds(lo, hi, cls, ref, rel=rel))


def test_full_in_device_memory_several_passes(sra):
    """600 boxes of the 3-[256]x4-1 net in FP64 (4.2 MB of state per box):
    the 1 GiB scratch of a pass holds 255 boxes, so three passes, the last
    one ragged."""
    mlp = WIDE["relu256x4"][0]()
    c, h = wl.make_boxes(600, seed=19, hw_lo=1 / 512, hw_hi=1 / 32)
    lo, hi, cls = run_boxes(sra, mlp, c, h, arith="full", precision="fp64")
    ref = oracle.bound_boxes(mlp, c, h, "full")
    assert_parity(compare_bounds(lo, hi, cls, ref, rel=FP64_REL))


def test_full_in_device_memory_contains_samples(sra):
    mlp = WIDE["elu_pe2_128x3"][0]()
    c, h = wl.make_boxes(48, seed=21, hw_lo=1 / 256, hw_hi=1 / 64)
    lo, hi, cls = run_boxes(sra, mlp, c, h, arith="full")
    for i in range(len(c)):
        f = forward(mlp, box_samples(c[i], h[i], n_grid=4, n_rand=128, seed=i))
        scale = abs(lo[i]) + abs(hi[i])
        assert f.min() >= lo[i] - 1e-5 * scale and f.max() <= hi[i] + 1e-5 * scale


def test_full_in_device_memory_octree_round(sra):
    """One round of Proc. 3 with affine-full on the 128-wide ReLU net and the
    FP64 re-check at band 1, which flags every node (|y0 - rad| <= |y0| +
    rad): the FP64 pass runs over the whole device-side list."""
    mlp = WIDE["relu128x3"][0]()
    net = sra.Net(mlp)
    nodes = wl.random_nodes(777, level=5, seed=23)
    fr = sra.nodes_to_tensor(nodes)
    out, leaves, counts = sra.classify_and_split(net, fr, 6, arith="full", recheck=True, recheck_band=1.0)
    torch.cuda.synchronize()
    cnt = counts.cpu().numpy()
    cls_ref, lo_ref, hi_ref, _ = oracle.classify_nodes(mlp, nodes, (-1, -1, -1), (1, 1, 1), oracle.OCTREE,
                                                       "full")
    scale = 0.5 * (np.abs(lo_ref + hi_ref) + (hi_ref - lo_ref))
    near = np.minimum(np.abs(lo_ref), np.abs(hi_ref)) <= 1e-6 * (1.0 + scale)
    for code, slot in ((1, 2), (2, 3)):
        sure = int(np.sum((cls_ref == code) & ~near))
        assert sure <= cnt[slot] <= sure + int(near.sum()), (code, cnt, sure, int(near.sum()))
    assert cnt[2] + cnt[3] + cnt[4] == len(nodes)
    assert cnt[0] == 8 * cnt[4] and cnt[5] == len(nodes)
    net.close()


def test_full_in_device_memory_tighter_than_truncate(sra):
    mlp = WIDE["relu256x4"][0]()
    c, h = wl.make_boxes(256, seed=25, hw_lo=1 / 256, hw_hi=1 / 16)
    lo_f, hi_f, _ = run_boxes(sra, mlp, c, h, arith="full")
    lo_t, hi_t, _ = run_boxes(sra, mlp, c, h, arith="truncate", K=64)
    assert np.mean(hi_f - lo_f) < np.mean(hi_t - lo_t)
