"""The benchmark's headline workload at its full size, in the launch
configuration the benchmark times: one octree round (Proc. 3) over 131,072
level-7 frontier nodes of the ReLU 3-[256]x8-1 network (the first 131,072
children of the UNKNOWN level-6 nodes of its FP32 octree), affine-truncate
K = 64 (Sec. 3.3), in BF16-sound with the FP64 re-check (band 1e-5) and in
FP32. One call bounds every node (one persistent CTA per SM).

The oracle cannot bound 131,072 nodes of this network in seconds, so outputs
are checked on a sample it computes node by node, and by properties that
hold at any size: each class is the sign test of its own range, the round's
counts equal the per-node classes, every UNKNOWN node below the last level
has eight children, and sampled values of f lie inside the BF16-sound range.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_02444_gb300 import workloads as wl
from tests.np_forward import box_samples, forward
from tests.parity import assert_parity, compare_bounds
from tests.sound_emulation import node_boxes

pytestmark = pytest.mark.gpu

B = 131072
LEVEL = 7
K = 64


@pytest.fixture(scope="module")
def sra():
    from paper_2202_02444_gb300 import sra as s
    return s


@pytest.fixture(scope="module")
def case(sra):
    mlp = wl.net_relu256x8()
    net = sra.Net(mlp)
    o32 = sra.make_opts(arith="truncate", K=K)
    leaves, _ = sra.extract_leaves(net, LEVEL - 1, opts=o32)
    kids, _, cnt = sra.classify_and_split(net, leaves, LEVEL, opts=o32)
    torch.cuda.synchronize()
    nk = int(cnt[sra.CNT_CHILDREN])
    assert nk > 0
    fr = kids[:nk].repeat((B + nk - 1) // nk, 1)[:B].contiguous()
    nodes = sra.tensor_to_nodes(fr)
    assert np.all(nodes["level"] == LEVEL)
    c, h = node_boxes(nodes)
    yield mlp, net, fr, nodes, c.astype(np.float32), h.astype(np.float32), min(nk, B)
    net.close()


def bound_all(sra, net, c, h, **kw):
    lo, hi, cls = sra.bound_boxes(net, torch.from_numpy(c).cuda(), torch.from_numpy(h).cuda(), **kw)
    sra.sync_status(net)
    return lo.cpu().numpy().astype(np.float64), hi.cpu().numpy().astype(np.float64), cls.cpu().numpy()


def sample(nk):
    """Distinct frontier nodes spread over the batch, and its last node."""
    idx = wl.sample_rows(nk, min(nk, 160), seed=17)
    return np.unique(np.concatenate([idx, [B - 1]]))


@pytest.mark.parametrize("precision", ["bf16_sound", "fp32"])
def test_round_counts_equal_node_classes(sra, case, precision):
    """The timed call (sra_classify_and_split on 131,072 nodes, up to level
    10) against sra_bound_boxes on the same nodes' boxes with the same
    options: identical classes, and the round's bookkeeping."""
    mlp, net, fr, nodes, c, h, nk = case
    opts = dict(arith="truncate", K=K, precision=precision, recheck=True, recheck_band=1e-5)
    out = torch.empty((8 * B, 4), dtype=torch.int16, device="cuda")
    leaves = torch.empty((B, 4), dtype=torch.int16, device="cuda")
    counts = torch.zeros(sra.CNT_N, dtype=torch.int64, device="cuda")
    sra.classify_and_split(net, fr, LEVEL + 3, opts=sra.make_opts(**opts), out=out, leaves=leaves, counts=counts)
    sra.sync_status(net)
    cnt = counts.cpu().numpy()
    lo, hi, cls = bound_all(sra, net, c, h, **opts)
    assert cnt[sra.CNT_POSITIVE] == np.sum(cls == 1)
    assert cnt[sra.CNT_NEGATIVE] == np.sum(cls == 2)
    assert cnt[sra.CNT_UNKNOWN] == np.sum(cls == 0)
    assert cnt[sra.CNT_CHILDREN] == 8 * cnt[sra.CNT_UNKNOWN]
    assert cnt[sra.CNT_LEAVES] == 0
    # each class is the sign test of the node's own range (re-checked nodes
    # carry their FP64 class and range)
    assert np.array_equal(cls, np.where(lo > 0, 1, np.where(hi < 0, 2, 0)))
    # the children are the octants of the UNKNOWN nodes, in frontier order
    kids = sra.tensor_to_nodes(out[:int(cnt[sra.CNT_CHILDREN])])
    par = nodes[cls == 0]
    assert np.all(kids["level"] == LEVEL + 1)
    assert np.array_equal(kids["ix"].reshape(-1, 8).min(1) // 2, par["ix"])
    assert np.array_equal(kids["iz"].reshape(-1, 8).max(1) // 2, par["iz"])
    print(f"{precision}: pos {cnt[2]} neg {cnt[3]} unk {cnt[4]} rechecked {cnt[5]} of {B}")


def test_fp32_full_frontier_sampled_parity(sra, case):
    """FP32 on all 131,072 nodes; a sample against the FP64 oracle within
    the FP32 tolerance (1e-5 of |c| + r), classes equal off the zero band."""
    mlp, net, fr, nodes, c, h, nk = case
    lo, hi, cls = bound_all(sra, net, c, h, arith="truncate", K=K)
    idx = sample(nk)
    ref = oracle.bound_boxes(mlp, c[idx], h[idx], "truncate", K=K)
    assert_parity(compare_bounds(lo[idx], hi[idx], cls[idx], ref))


def test_bf16_sound_full_frontier_sampled(sra, case):
    """BF16-sound on all 131,072 nodes. On the sample: every value of f at
    dense points of the node lies inside [lo, hi] (no tolerance); the range
    contains the oracle's (selection near-ties exempt); no decided class
    contradicts the oracle."""
    mlp, net, fr, nodes, c, h, nk = case
    lo, hi, cls = bound_all(sra, net, c, h, arith="truncate", K=K, precision="bf16_sound")
    assert np.all(hi >= lo)
    idx = sample(nk)
    ref = oracle.bound_boxes(mlp, c[idx], h[idx], "truncate", K=K)
    tie = ref["sel_gap"] < 1e-2
    assert np.all(((lo[idx] <= ref["lo"]) & (hi[idx] >= ref["hi"])) | tie)
    s = cls[idx]
    assert not np.any(((s == 1) & (ref["cls"] == 2)) | ((s == 2) & (ref["cls"] == 1)))
    for j, i in enumerate(idx):
        f = forward(mlp, box_samples(c[i], h[i], n_grid=3, n_rand=32, seed=int(i)))
        assert f.min() >= lo[i] and f.max() <= hi[i], (i, f.min(), f.max(), lo[i], hi[i])
