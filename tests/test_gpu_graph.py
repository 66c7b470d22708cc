"""The asynchronous entry points inside captured CUDA graphs.

sra_bound_boxes, sra_classify_and_split, sra_classify_and_split_batch and
sra_cast_rays only enqueue work on the caller's stream: kernels (the batched
round's segment tables travel as kernel parameters), memsets and
stream-ordered scratch. They can therefore be captured into a CUDA graph and
replayed with new inputs written into the same buffers. A replay must give
the same results, bit for bit, as an eager call on the same inputs. The
entry points that read counts back to the host between their launches
refuse a capturing stream.
"""
import numpy as np
import pytest
import torch

from paper_2202_02444_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sra():
    from paper_2202_02444_gb300 import sra as s
    return s


def capture(fn):
    """Warm up fn on a side stream, then capture it; returns the graph."""
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    torch.cuda.synchronize()
    return g


@pytest.mark.parametrize("precision", ["fp32", "bf16_sound"])
def test_bound_boxes_graph_replay(sra, precision):
    net = sra.Net(wl.net_relu256x8())
    opts = sra.make_opts(arith="truncate", K=64, precision=precision, recheck=True, recheck_band=1e-5)
    n = 1000
    c = torch.empty((n, 3), device="cuda")
    h = torch.empty((n, 3), device="cuda")
    lo = torch.empty(n, device="cuda")
    hi = torch.empty(n, device="cuda")
    cl = torch.empty(n, dtype=torch.uint8, device="cuda")
    c0, h0 = wl.make_boxes(n, seed=1, hw_hi=1 / 16)
    c.copy_(torch.from_numpy(c0))
    h.copy_(torch.from_numpy(h0))
    g = capture(lambda: sra.bound_boxes(net, c, h, opts=opts, lo=lo, hi=hi, cls=cl))
    for seed in (2, 3):
        c1, h1 = wl.make_boxes(n, seed=seed, hw_hi=1 / 16)
        c.copy_(torch.from_numpy(c1))
        h.copy_(torch.from_numpy(h1))
        g.replay()
        torch.cuda.synchronize()
        got = (lo.clone(), hi.clone(), cl.clone())
        ref = sra.bound_boxes(net, c, h, opts=opts)
        torch.cuda.synchronize()
        for a, b in zip(got, ref):
            assert torch.equal(a, b)
    net.close()


def test_classify_and_split_graph_replay(sra):
    net = sra.Net(wl.net_small_relu())
    opts = sra.make_opts(arith="fixed", recheck=True, recheck_band=1e-5)
    n = 777
    fr = torch.empty((n, 4), dtype=torch.int16, device="cuda")
    out = torch.empty((8 * n, 4), dtype=torch.int16, device="cuda")
    leaves = torch.empty((n, 4), dtype=torch.int16, device="cuda")
    counts = torch.zeros(sra.CNT_N, dtype=torch.int64, device="cuda")
    fr.copy_(sra.nodes_to_tensor(wl.random_nodes(n, level=5, seed=1)))

    def round_():
        counts.zero_()
        sra.classify_and_split(net, fr, 6, opts=opts, out=out, leaves=leaves, counts=counts)

    g = capture(round_)
    for seed in (2, 3):
        fr.copy_(sra.nodes_to_tensor(wl.random_nodes(n, level=5, seed=seed)))
        g.replay()
        torch.cuda.synchronize()
        cnt = counts.clone()
        kids = out[:int(cnt[sra.CNT_CHILDREN])].clone()
        out2, _, cnt2 = sra.classify_and_split(net, fr, 6, opts=opts)
        torch.cuda.synchronize()
        assert torch.equal(cnt, cnt2)
        assert torch.equal(kids, out2[:int(cnt2[sra.CNT_CHILDREN])])
    net.close()


def test_capture_refused_where_host_data_moves(sra):
    """sra_extract_leaves reads each level's counts back to the host before
    it launches the next level: inside a stream capture it returns
    SRA_EUNSUPPORTED and enqueues nothing. Outside a capture it runs as
    usual."""
    net = sra.Net(wl.net_small_relu())
    opts = sra.make_opts(arith="truncate", K=16)
    codes = []
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        try:
            sra.extract_leaves(net, 3, opts=opts)
            codes.append(0)
        except sra.SraError as e:
            codes.append(e.code)
    torch.cuda.synchronize()
    assert codes == [sra.EUNSUPPORTED]
    lv, lc = sra.extract_leaves(net, 3, opts=opts)
    torch.cuda.synchronize()
    assert int(lc.sum()) > 0
    net.close()


def test_batch_round_graph_replay(sra):
    """The batched round over two networks (an FP32 SIMT segment beside a
    BF16-sound tensor-core one), captured into a graph and replayed on new
    frontier nodes in the same buffers, gives what an eager round gives on
    those nodes, bit for bit: classes, children, leaves and counters."""
    nets = [sra.Net(wl.net_small_relu()), sra.Net(wl.make_mlp([128] * 3, "relu", seed=50))]
    opts = [sra.make_opts(arith="truncate", K=16),
            sra.make_opts(arith="truncate", K=16, precision="bf16_sound")]
    n0, n1 = 300, 200
    segs = [dict(net=0, max_level=6, first=0, n=n0, out_first=0, cap_out=8 * n0, leaf_first=0, cap_leaves=n0),
            dict(net=1, max_level=5, first=n0, n=n1, out_first=8 * n0, cap_out=8 * n1, leaf_first=n0,
                 cap_leaves=n1)]

    def nodes(seed):
        return sra.nodes_to_tensor(np.concatenate([wl.random_nodes(n0, level=5, seed=seed),
                                                   wl.random_nodes(n1, level=4, seed=seed + 100)]))

    fr = torch.empty((n0 + n1, 4), dtype=torch.int16, device="cuda")
    out = torch.empty((8 * (n0 + n1), 4), dtype=torch.int16, device="cuda")
    leaves = torch.empty((n0 + n1, 4), dtype=torch.int16, device="cuda")
    counts = torch.zeros((2, sra.CNT_N), dtype=torch.int64, device="cuda")
    fr.copy_(nodes(1))

    def round_():
        counts.zero_()
        out.fill_(-1)
        leaves.fill_(-1)
        sra.classify_and_split_batch(nets, opts, fr, segs, out, leaves, counts=counts)

    g = capture(round_)
    for seed in (2, 3):
        fr.copy_(nodes(seed))
        g.replay()
        torch.cuda.synchronize()
        got = (counts.clone(), out.clone(), leaves.clone())
        out2 = torch.full_like(out, -1)
        leaves2 = torch.full_like(leaves, -1)
        cnt2 = sra.classify_and_split_batch(nets, opts, fr, segs, out2, leaves2)
        torch.cuda.synchronize()
        assert torch.equal(got[0], cnt2)
        assert torch.equal(got[1], out2) and torch.equal(got[2], leaves2)
        assert int(cnt2[:, sra.CNT_CHILDREN].sum()) > 0
    for n in nets:
        sra.sync_status(n)
        n.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16_sound"])
def test_cast_rays_graph_replay(sra, precision):
    mlp = wl.net_small_relu() if precision == "fp32" else wl.make_mlp([128] * 3, "elu", seed=35, pe_octaves=2)
    net = sra.Net(mlp)
    opts = sra.make_opts(arith="fixed", delta=1e-3, precision=precision, max_iters=3000)
    n = 300
    o = torch.empty((n, 3), device="cuda")
    d = torch.empty((n, 3), device="cuda")
    t = torch.empty(n, device="cuda")
    it = torch.empty(n, dtype=torch.int32, device="cuda")
    o0, d0 = wl.sphere_rays(n, seed=1, radius=2.0)
    o.copy_(torch.from_numpy(o0))
    d.copy_(torch.from_numpy(d0))
    g = capture(lambda: sra.cast_rays(net, o, d, opts=opts, t_hit=t, iters=it))
    o1, d1 = wl.sphere_rays(n, seed=2, radius=2.0)
    o.copy_(torch.from_numpy(o1))
    d.copy_(torch.from_numpy(d1))
    g.replay()
    torch.cuda.synchronize()
    got_t, got_it = t.clone(), it.clone()
    t2, it2 = sra.cast_rays(net, o, d, opts=opts)
    torch.cuda.synchronize()
    assert torch.equal(torch.nan_to_num(got_t, nan=-1.0), torch.nan_to_num(t2, nan=-1.0))
    assert torch.equal(got_it, it2)
    assert np.isfinite(got_t.cpu().numpy()).any()
    net.close()
