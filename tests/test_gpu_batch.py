"""The batched round over many networks (sra_classify_and_split_batch):
every segment's classes, children, leaves and counters equal a lone
sra_classify_and_split call on that segment (Proc. 3)."""
import numpy as np
import pytest
import torch

from paper_2202_02444_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sra():
    from paper_2202_02444_gb300 import sra as s
    return s


def setup(sra, specs, seed=0):
    """specs: (mlp, opts kwargs, level, n_nodes, max_level) per network."""
    nets, opts, fr, segs = [], [], [], []
    first = out_first = leaf_first = 0
    for j, (mlp, kw, level, n, max_level) in enumerate(specs):
        nets.append(sra.Net(mlp))
        opts.append(sra.make_opts(**kw))
        nodes = wl.random_nodes(n, level, seed=seed + j) if n else np.zeros(0, wl.NODE_DTYPE)
        if kw.get("split") == "kd":  # octree level L is k-d level 3L on the cube root
            nodes["level"] = 3 * level
        fr.append(nodes)
        fan = 8 if kw.get("split", "octree") == "octree" else 2
        segs.append(dict(net=j, max_level=max_level, first=first, n=n, out_first=out_first,
                         cap_out=n * fan, leaf_first=leaf_first, cap_leaves=n))
        first += n
        out_first += n * fan
        leaf_first += n
    frontier = sra.nodes_to_tensor(np.concatenate(fr)) if first else torch.zeros((1, 4), dtype=torch.int16,
                                                                                  device="cuda")
    out = torch.full((max(out_first, 1), 4), -1, dtype=torch.int16, device="cuda")
    leaves = torch.full((max(leaf_first, 1), 4), -1, dtype=torch.int16, device="cuda")
    return nets, opts, frontier, segs, out, leaves


def check_against_lone(sra, nets, opts, frontier, segs, out, leaves, counts):
    cnt = counts.cpu().numpy()
    for k, sg in enumerate(segs):
        a, n = sg["first"], sg["n"]
        net, o = nets[sg["net"]], opts[sg["net"]]
        ref_out, ref_leaves, ref_cnt = sra.classify_and_split(
            net, frontier[a:a + n] if n else frontier[:0], sg["max_level"], opts=o,
            cap_out=sg["cap_out"], cap_leaves=sg["cap_leaves"])
        rc = ref_cnt.cpu().numpy()
        assert np.array_equal(cnt[k], rc), (k, cnt[k], rc)
        nc = min(int(rc[0]), sg["cap_out"])
        nl = min(int(rc[1]), sg["cap_leaves"])
        got = out[sg["out_first"]:sg["out_first"] + nc].cpu().numpy()
        assert np.array_equal(got, ref_out[:nc].cpu().numpy()), k
        gl = leaves[sg["leaf_first"]:sg["leaf_first"] + nl].cpu().numpy()
        assert np.array_equal(gl, ref_leaves[:nl].cpu().numpy()), k


def test_batch_equals_lone_rounds(sra):
    specs = [
        (wl.net_small_relu(), dict(arith="fixed"), 3, 300, 7),
        (wl.make_mlp([64] * 5, "sin", seed=61), dict(arith="truncate", K=16), 4, 1500, 8),
        (wl.make_mlp([128] * 3, "elu", seed=62), dict(arith="truncate", K=32, block_threads=512), 5, 2048, 5),
        (wl.make_mlp([256] * 4, "relu", seed=63), dict(arith="truncate", K=64), 4, 777, 9),
        (wl.make_mlp([512] * 3, "elu", seed=64), dict(arith="truncate", K=16), 3, 129, 6),
        (wl.make_mlp([96, 96], "relu", seed=65, pe_octaves=2), dict(arith="fixed"), 2, 50, 2),
        (wl.make_mlp([32] * 3, "relu", seed=66), dict(arith="interval"), 6, 4000, 6),
    ]
    nets, opts, frontier, segs, out, leaves = setup(sra, specs)
    try:
        counts = sra.classify_and_split_batch(nets, opts, frontier, segs, out, leaves)
        torch.cuda.synchronize()
        check_against_lone(sra, nets, opts, frontier, segs, out, leaves, counts)
        # segments at their max level emitted leaves
        cnt = counts.cpu().numpy()
        assert cnt[2][1] > 0 and cnt[5][1] > 0 and cnt[6][1] > 0
    finally:
        for n in nets:
            n.close()


def test_batch_kd_split_empty_and_overflow(sra):
    specs = [
        (wl.make_mlp([64] * 3, "relu", seed=70), dict(arith="truncate", K=8, split="kd"), 2, 900, 20),
        (wl.make_mlp([64] * 3, "elu", seed=71), dict(arith="fixed"), 3, 0, 5),   # empty segment
        (wl.make_mlp([128] * 3, "relu", seed=72), dict(arith="fixed"), 4, 600, 8),
    ]
    nets, opts, frontier, segs, out, leaves = setup(sra, specs, seed=5)
    segs[2]["cap_out"] = 100  # far fewer than the children: the rest is counted, not written
    try:
        counts = sra.classify_and_split_batch(nets, opts, frontier, segs, out, leaves)
        torch.cuda.synchronize()
        check_against_lone(sra, nets, opts, frontier, segs, out, leaves, counts)
        cnt = counts.cpu().numpy()
        assert cnt[2][0] > 100
        assert not cnt[1].any()
        # nothing was written past the overflowing segment's capacity
        tail = out[segs[2]["out_first"] + 100:].cpu().numpy()
        assert (tail == -1).all()
    finally:
        for n in nets:
            n.close()


def test_batch_appends_to_counts(sra):
    """Chunked calls append after the counts already present."""
    specs = [(wl.make_mlp([64] * 3, "relu", seed=80), dict(arith="fixed"), 4, 1000, 8)]
    nets, opts, frontier, segs, out, leaves = setup(sra, specs)
    try:
        half = [dict(segs[0], n=500, cap_out=8000), dict(segs[0], first=500, n=500, cap_out=8000)]
        c = sra.classify_and_split_batch(nets, opts, frontier, [half[0]], out, leaves)
        half[1]["out_first"] = 0
        c = sra.classify_and_split_batch(nets, opts, frontier, [half[1]], out, leaves, counts=c)
        ref_out, _, ref_cnt = sra.classify_and_split(nets[0], frontier, 8, opts=opts[0])
        torch.cuda.synchronize()
        rc = ref_cnt.cpu().numpy()
        assert np.array_equal(c.cpu().numpy()[0], rc)
        assert np.array_equal(out[:rc[0]].cpu().numpy(), ref_out[:rc[0]].cpu().numpy())
    finally:
        nets[0].close()


def test_batch_bf16_segments_equal_lone_rounds(sra):
    """Segments in BF16-sound and plain BF16 (their ReLU, ELU and sin
    networks have the tensor-core path) run beside FP32 segments in one batched round; each
    equals a lone round with the same options."""
    specs = [
        (wl.make_mlp([128] * 4, "relu", seed=31), dict(arith="truncate", K=64, precision="bf16_sound"), 4, 1001, 6),
        (wl.net_small_relu(), dict(arith="truncate", K=16), 3, 500, 7),
        (wl.make_mlp([256] * 3, "relu", seed=32), dict(arith="truncate", K=64, precision="bf16"), 5, 777, 5),
        (wl.make_mlp([256] * 5, "relu", seed=33), dict(arith="truncate", K=64, precision="bf16_sound"), 3, 3, 9),
        (wl.make_mlp([64] * 4, "elu", seed=34), dict(arith="fixed"), 4, 900, 8),
        (wl.make_mlp([128] * 3, "elu", seed=35), dict(arith="truncate", K=64, precision="bf16_sound"), 4, 640, 7),
        (wl.make_mlp([256] * 3, "sin", seed=39), dict(arith="truncate", K=64, precision="bf16_sound"), 6, 513, 9),
        (wl.make_mlp([128] * 4, "sin", seed=41), dict(arith="truncate", K=64, precision="bf16"), 5, 300, 8),
        (wl.make_mlp([512] * 3, "relu", seed=42), dict(arith="truncate", K=64, precision="bf16_sound"), 4, 301, 7),
        (wl.make_mlp([512] * 4, "elu", seed=47), dict(arith="truncate", K=64, precision="bf16"), 3, 64, 6),
        (wl.make_mlp([256] * 4, "relu", seed=48), dict(arith="truncate", K=16, precision="bf16_sound"), 4, 700, 7),
        (wl.make_mlp([128] * 5, "sin", seed=49), dict(arith="truncate", K=32, precision="bf16"), 4, 333, 7),
        (wl.make_mlp([256] * 3, "elu", seed=50), dict(arith="truncate", K=128, precision="bf16_sound"), 4, 257, 6),
        # widths 64 and 32 on the 128-wide kernel with zero-padded weights
        (wl.make_mlp([64] * 5, "relu", seed=51), dict(arith="truncate", K=16, precision="bf16_sound"), 4, 450, 7),
        (wl.make_mlp([32] * 3, "sin", seed=52), dict(arith="truncate", K=32, precision="bf16"), 5, 200, 7),
        (wl.make_mlp([96, 200, 64], "relu", seed=53), dict(arith="truncate", K=64, precision="bf16_sound"), 4, 350,
         7),
    ]
    nets, opts, frontier, segs, out, leaves = setup(sra, specs, seed=9)
    try:
        counts = sra.classify_and_split_batch(nets, opts, frontier, segs, out, leaves)
        for n in nets:
            sra.sync_status(n)
        check_against_lone(sra, nets, opts, frontier, segs, out, leaves, counts)
        cnt = counts.cpu().numpy()
        assert cnt[2][1] > 0  # the BF16 segment at its max level emitted leaves
    finally:
        for n in nets:
            n.close()


def test_batch_rejects_unserved_bf16(sra):
    """BF16 segments need the tensor-core path (3 inputs, hidden widths up to
    512, all ReLU, all ELU or all sin) and affine-truncate K = 16, 32, 64 or
    128; FP64 and re-checks are not batched."""
    net = sra.Net(wl.make_mlp([128] * 3, "relu", seed=1, pe_octaves=1))  # encoded input: no tensor-core path
    net2 = sra.Net(wl.make_mlp([128] * 3, "relu", seed=1))
    try:
        fr = sra.nodes_to_tensor(wl.random_nodes(10, 3))
        out = torch.empty((80, 4), dtype=torch.int16, device="cuda")
        seg = [dict(net=0, max_level=5, n=10, cap_out=80, cap_leaves=0)]
        for n, o in ((net, sra.make_opts(arith="truncate", K=64, precision="bf16_sound")),
                     (net2, sra.make_opts(arith="truncate", K=48, precision="bf16_sound")),  # K in {16, 32, 64, 128}
                     (net2, sra.make_opts(arith="truncate", K=64, precision="fp64")),
                     (net2, sra.make_opts(arith="truncate", K=64, precision="bf16", recheck=True))):
            with pytest.raises(sra.SraError) as e:
                sra.classify_and_split_batch([n], [o], fr, seg, out, out)
            assert e.value.code == sra.EUNSUPPORTED
    finally:
        net.close()
        net2.close()
