"""The request loop (sra_serve): every result in a concurrent mix equals the
result of a lone call of the entry point it uses; admission by frontier
memory; per-request failures stay with their request."""
import numpy as np
import pytest
import torch

from paper_2202_02444_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sra():
    from paper_2202_02444_gb300 import sra as s
    return s


@pytest.fixture(scope="module")
def nets(sra):
    mlps = [wl.net_small_relu(),
            wl.make_mlp([128] * 3, "relu", seed=50),
            wl.make_mlp([128] * 3, "elu", seed=51, pe_octaves=2),
            wl.make_mlp([64] * 4, "sin", seed=52)]
    ns = [sra.Net(m) for m in mlps]
    yield ns
    for n in ns:
        n.close()


def forms(sra):
    return [sra.make_opts(arith="fixed", delta=1e-3, max_iters=300),              # 0: FP32 fixed
            sra.make_opts(arith="truncate", K=16),                                # 1: FP32 truncate
            sra.make_opts(arith="fixed", precision="bf16", delta=1e-3, max_iters=300),  # 2: BF16 rays
            sra.make_opts(arith="fixed", precision="bf16_sound", delta=1e-3, max_iters=300)]  # 3: BF16-sound rays


def make_trace(sra, n_req, seed, spacing=0.0):
    """Seeded mix of ray tiles, box batches and leaf jobs; returns the
    requests and the tensors they point to (inputs and outputs)."""
    rng = np.random.default_rng(seed)
    reqs, bufs = [], []
    for i in range(n_req):
        kind = i % 3
        net = int(rng.integers(0, 4))
        arrival = i * spacing
        if kind == sra.REQ_RAYS:
            n = int(rng.integers(100, 1500))
            o, d = wl.sphere_rays(n, seed=100 + i, radius=2.0)
            o, d = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
            t = torch.full((n,), -7.0, device="cuda")
            it = torch.full((n,), -7, dtype=torch.int32, device="cuda")
            u = rng.random()
            form = (2 if u < 0.25 else 3) if net in (1, 2) and u < 0.5 else 0
            reqs.append(sra.ray_request(net, form, arrival, o, d, t, it))
            bufs.append(("rays", net, form, (o, d), (t, it)))
        elif kind == sra.REQ_BOXES:
            n = int(rng.integers(256, 4096))
            c, h = wl.make_boxes(n, seed=200 + i)
            c, h = torch.from_numpy(c).cuda(), torch.from_numpy(h).cuda()
            lo = torch.full((n,), -7.0, device="cuda")
            hi = torch.full((n,), -7.0, device="cuda")
            cl = torch.full((n,), 9, dtype=torch.uint8, device="cuda")
            form = int(rng.integers(0, 2))
            reqs.append(sra.box_request(net, form, arrival, c, h, lo, hi, cl))
            bufs.append(("boxes", net, form, (c, h), (lo, hi, cl)))
        else:
            depth = int(rng.integers(3, 6))
            leaves = torch.full((1 << 16, 4), -1, dtype=torch.int16, device="cuda")
            form = int(rng.integers(0, 2))
            reqs.append(sra.leaf_request(net, form, arrival, depth, leaves))
            bufs.append(("leaves", net, form, depth, leaves))
    return reqs, bufs


def alone(sra, nets, fo, b):
    """The same query as a lone call of its entry point."""
    kind, net, form = b[0], nets[b[1]], fo[b[2]]
    if kind == "rays":
        t, it = sra.cast_rays(net, *b[3], opts=form)
        return t, it
    if kind == "boxes":
        lo, hi, cl = sra.bound_boxes(net, *b[3], opts=form)
        return lo, hi, cl
    leaves, _ = sra.extract_leaves(net, b[3], opts=form)
    return (leaves,)


def same(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return a.shape == b.shape and np.array_equal(a, b, equal_nan=a.dtype.kind == "f")


def test_mix_equals_alone(sra, nets):
    fo = forms(sra)
    reqs, bufs = make_trace(sra, 24, seed=1)
    out = sra.serve(nets, fo, reqs, slots=4, frontier_bytes=64 << 20, realtime=False)
    torch.cuda.synchronize()
    assert all(r.status == 0 for r in out), [(i, r.status) for i, r in enumerate(out) if r.status]
    assert len({r.slot for r in out}) > 1  # the mix really used several slots
    # requests overlapped in time
    spans = sorted((r.t_admit, r.t_done) for r in out)
    assert any(spans[k + 1][0] < spans[k][1] for k in range(len(spans) - 1))
    for r, b in zip(out, bufs):
        ref = alone(sra, nets, fo, b)
        torch.cuda.synchronize()
        if b[0] == "leaves":
            n = r.n_out
            assert n == ref[0].shape[0], (n, ref[0].shape)
            assert same(b[4][:n], ref[0])
            assert r.levels >= 1
        else:
            for got, want in zip(b[4], ref):
                assert same(got, want), b[0]


def test_admission_by_frontier_memory(sra, nets):
    """A budget that holds one leaf job at a time: leaf jobs never overlap."""
    fo = forms(sra)
    cap = 1 << 14
    per_job = (4 + 1) * (((cap * 8) + 255) // 256 * 256) + 256  # one buffer per level 0..4
    reqs, keep = [], []
    for i in range(3):
        leaves = torch.empty((cap, 4), dtype=torch.int16, device="cuda")
        keep.append(leaves)
        reqs.append(sra.leaf_request(i % 2, 0, 0.0, 4, leaves))
    out = sra.serve(nets, fo, reqs, slots=4, frontier_bytes=per_job + 1024, realtime=False)
    assert all(r.status == 0 for r in out)
    spans = sorted((r.t_admit, r.t_done) for r in out)
    for k in range(len(spans) - 1):
        assert spans[k + 1][0] >= spans[k][1]


@pytest.mark.parametrize("net_i,depth,split", [(0, 6, "octree"), (1, 5, "octree"), (0, 15, "kd")])
def test_leaf_job_levels_larger_than_its_buffers(sra, nets, net_i, depth, split):
    """A leaf job whose tree has levels larger than its per-level buffers
    walks them in chunks, depth-first, and still returns the leaves of a
    level-by-level build in the same order."""
    fo = forms(sra) + [sra.make_opts(arith="truncate", K=16, split=split)]
    form = len(fo) - 1
    ref, lc = sra.extract_leaves(nets[net_i], depth, opts=fo[form])
    n = ref.shape[0]
    widest = int(lc.sum(axis=1).max())
    cap = max(n, 64)
    assert widest > cap, (widest, cap)  # a level-by-level job with this cap overflows
    leaves = torch.full((cap, 4), -1, dtype=torch.int16, device="cuda")
    req = sra.leaf_request(net_i, form, 0.0, depth, leaves)
    out = sra.serve(nets, fo, [req], slots=1, frontier_bytes=64 << 20, realtime=False)
    assert out[0].status == 0, out[0].status
    assert out[0].n_out == n and out[0].levels == depth + 1
    assert same(leaves[:n], ref)


def test_leaf_job_stops_when_its_leaves_overflow(sra, nets):
    fo = forms(sra)
    ref, _ = sra.extract_leaves(nets[0], 6, opts=fo[1])
    cap = ref.shape[0] // 3
    leaves = torch.full((cap, 4), -1, dtype=torch.int16, device="cuda")
    out = sra.serve(nets, fo, [sra.leaf_request(0, 1, 0.0, 6, leaves)], slots=1,
                    frontier_bytes=64 << 20, realtime=False)
    assert out[0].status == sra.ECAPACITY
    assert cap < out[0].n_out <= ref.shape[0]
    assert same(leaves, ref[:cap])  # the first cap leaves, in order


def test_request_failures_stay_local(sra, nets):
    # form 4: BF16 rays in affine-truncate, which the tensor-core ray kernel
    # does not serve (it marches affine-fixed segments)
    fo = forms(sra) + [sra.make_opts(arith="truncate", K=4, precision="bf16", delta=1e-3, max_iters=300)]
    o, d = wl.sphere_rays(64, seed=3, radius=2.0)
    o, d = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    t = torch.empty(64, device="cuda")
    small = torch.empty((4, 4), dtype=torch.int16, device="cuda")  # too small for level 1
    big = torch.empty((1 << 20, 4), dtype=torch.int16, device="cuda")  # reservation > budget
    t_ok = torch.empty(64, device="cuda")
    reqs = [sra.ray_request(3, 4, 0.0, o, d, t),        # BF16 truncate rays: unsupported
            sra.leaf_request(0, 0, 0.0, 3, small),
            sra.leaf_request(1, 0, 0.0, 3, big),
            sra.ray_request(0, 0, 0.0, o, d, t_ok)]
    out = sra.serve(nets, fo, reqs, slots=2, frontier_bytes=4 << 20, realtime=False)
    assert out[0].status == sra.EUNSUPPORTED
    assert out[1].status == sra.ECAPACITY and out[1].n_out > 4
    assert out[2].status == sra.ENOMEM and out[2].slot == -1
    assert out[3].status == 0
    ref, _ = sra.cast_rays(nets[0], o, d, opts=fo[0])
    assert same(t_ok, ref)


def test_realtime_arrivals(sra, nets):
    fo = forms(sra)
    reqs, bufs = make_trace(sra, 9, seed=2, spacing=0.03)
    out = sra.serve(nets, fo, reqs, slots=3, frontier_bytes=32 << 20, realtime=True)
    for r in out:
        assert r.status == 0
        assert r.t_admit >= r.arrival - 1e-6
        assert r.t_done >= r.t_admit
