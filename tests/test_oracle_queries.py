"""Pins for the oracle's geometric queries: BuildSpatialTree (Proc. 3, fixed
depth) and CastRay (Proc. 2), against analytic planes, brute-force grids and
the delta-convergence semantics of Sec. 4.1.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2202_02444_gb300 import workloads as wl
from tests.np_forward import forward

XL, XU = np.array([-1.0, -1.0, -1.0]), np.array([1.0, 1.0, 1.0])


def plane_net(n=(0.3, -0.5, 0.8), d=0.1):
    n = np.asarray(n, np.float64)
    return wl.make_custom_mlp([3, 1], [], [(n[None, :], np.array([-d]))])


def cells(level):
    m = 1 << level
    ii = np.arange(m)
    I = np.stack(np.meshgrid(ii, ii, ii, indexing="ij"), -1).reshape(-1, 3)
    w = 2.0 / m
    lo = -1.0 + I * w
    return I, lo, lo + w


def corner_values(net, lo, hi):
    cs = np.array([[a, b, c] for a in (0, 1) for b in (0, 1) for c in (0, 1)], float)
    pts = lo[:, None, :] + cs[None] * (hi - lo)[:, None, :]
    return forward(net, pts.reshape(-1, 3)).reshape(len(lo), 8)


def node_ranges(nodes, split):
    """Per-axis (lo, hi) of each node, replaying the widest-axis splits."""
    out = []
    for nd in nodes:
        lvl = int(nd["level"])
        if split == oracle.OCTREE:
            n3 = [lvl] * 3
        else:
            e, n3 = [2.0, 2.0, 2.0], [0, 0, 0]
            for _ in range(lvl):
                a = int(np.argmax(e))
                e[a] /= 2
                n3[a] += 1
        idx = [int(nd["ix"]), int(nd["iy"]), int(nd["iz"])]
        w = [2.0 / (1 << k) for k in n3]
        out.append([(-1 + idx[a] * w[a], -1 + (idx[a] + 1) * w[a]) for a in range(3)])
    return out


@pytest.mark.parametrize("split", [oracle.OCTREE, oracle.KD])
def test_tree_plane_exact_leaf_set(split):
    """For an affine f the affine bound is exact (Sec. 3.2), so the UNKNOWN
    leaves at the final depth are exactly the cells whose corners straddle 0
    (an octree depth D equals a k-d depth 3D on a cube, Sec. 4.7)."""
    net = plane_net()
    D = 4
    maxl = D if split == oracle.OCTREE else 3 * D
    nodes, counts = oracle.build_tree(net, XL, XU, maxl, split=split)
    unk = nodes[nodes["cls"] == oracle.UNKNOWN]
    assert np.all(unk["level"] == maxl)
    got = {(int(a), int(b), int(c)) for a, b, c in zip(unk["ix"], unk["iy"], unk["iz"])}
    I, lo, hi = cells(D)
    cv = corner_values(net, lo, hi)
    straddle = (cv.min(1) <= 0) & (cv.max(1) >= 0)
    want = {tuple(map(int, t)) for t in I[straddle]}
    assert got == want
    assert counts[0] + counts[1] + counts[2] == len(nodes)


@pytest.mark.parametrize("split", [oracle.OCTREE, oracle.KD])
def test_tree_partitions_domain_and_classes_hold(split):
    """Returned nodes tile the root box exactly once; POSITIVE/NEGATIVE nodes
    have all sampled values of the right strict sign (Sec. 4.5 guarantee)."""
    net = wl.net_small_relu()
    D = 4
    maxl = D if split == oracle.OCTREE else 3 * D
    nodes, _ = oracle.build_tree(net, XL, XU, maxl, split=split)
    rng = node_ranges(nodes, split)
    m = 1 << D
    cover = np.zeros((m, m, m), np.int32)
    g = np.random.default_rng(0)
    for nd, r in zip(nodes, rng):
        sl = tuple(slice(int(round((a + 1) / 2 * m)), int(round((b + 1) / 2 * m))) for a, b in r)
        cover[sl] += 1
        if nd["cls"] != oracle.UNKNOWN:
            lo = np.array([a for a, _ in r]); hi = np.array([b for _, b in r])
            pts = lo + g.uniform(0, 1, size=(16, 3)) * (hi - lo)
            ys = forward(net, pts)
            if nd["cls"] == oracle.POSITIVE:
                assert ys.min() > 0
            else:
                assert ys.max() < 0
    assert np.all(cover == 1)


@pytest.mark.parametrize("split", [oracle.OCTREE, oracle.KD])
def test_tree_leaves_cover_sign_changes(split):
    """Every finest-level cell whose corner samples change sign is an UNKNOWN
    leaf (no surface cell is missed; Sec. 4.7 'same output as brute force')."""
    net = wl.net_small_relu()
    D = 5
    maxl = D if split == oracle.OCTREE else 3 * D
    nodes, _ = oracle.build_tree(net, XL, XU, maxl, split=split)
    unk = nodes[nodes["cls"] == oracle.UNKNOWN]
    got = {(int(a), int(b), int(c)) for a, b, c in zip(unk["ix"], unk["iy"], unk["iz"])}
    I, lo, hi = cells(D)
    cv = corner_values(net, lo, hi)
    change = (cv.min(1) < 0) & (cv.max(1) > 0)
    need = {tuple(map(int, t)) for t in I[change]}
    assert need, "test net has no surface in the domain"
    assert need <= got


def test_ray_plane_analytic():
    """Proc. 2 on an affine f: the hit satisfies t < t* <= t + delta, with t*
    the analytic crossing; a ray moving away misses."""
    nvec = np.array([0.3, -0.5, 0.8])
    net = plane_net(nvec, 0.1)
    o, d = wl.sphere_rays(64, seed=3)
    delta = 1e-3
    r = oracle.cast_rays(net, o, d, "fixed", delta=delta)
    o64, d64 = o.astype(np.float64), d.astype(np.float64)
    n32 = nvec.astype(np.float32).astype(np.float64)
    d32 = float(np.float32(-0.1))
    tstar = -(o64 @ n32 + d32) / (d64 @ n32)
    for i in range(64):
        if 0 < tstar[i] < 10 - delta:
            assert r["status"][i] == 1
            assert r["t"][i] < tstar[i] + 1e-12 and tstar[i] <= r["t"][i] + delta + 1e-12
        elif tstar[i] < 0 or tstar[i] > 10 + delta:
            assert r["status"][i] == 0 and math.isinf(r["t"][i])


@pytest.mark.parametrize("arith", ["fixed", "truncate"])
def test_ray_delta_semantics_random_net(arith):
    """Sec. 4.1: the returned t has f(p + (t+delta) r) of the opposite sign to
    f(p); any sign change sampled on [0, t] is a feature thinner than delta
    (the sign comes back within delta)."""
    net = wl.net_small_relu()
    o, d = wl.sphere_rays(48, seed=5, radius=2.0)
    delta = 1e-3
    r = oracle.cast_rays(net, o, d, arith, K=8, delta=delta)
    assert (r["status"] == 1).sum() > 10
    for i in range(48):
        p, dv = o[i].astype(np.float64), d[i].astype(np.float64)
        f0 = forward(net, p[None])[0]
        if r["status"][i] == 1:
            t = r["t"][i]
            fc = forward(net, (p + (t + delta) * dv)[None])[0]
            assert (fc >= 0) != (f0 >= 0)
            tt = np.arange(0.0, t, delta / 4)
        else:
            assert r["status"][i] == 0
            tt = np.arange(0.0, 10.0, delta / 4)
        fs = forward(net, p[None] + tt[:, None] * dv[None])
        flip = np.nonzero((fs >= 0) != (f0 >= 0))[0]
        for j in flip:
            back = (fs[j:j + 5] >= 0) == (f0 >= 0)
            assert back.any(), (i, tt[j])


def test_ray_iteration_cap():
    net = wl.net_small_relu()
    o, d = wl.sphere_rays(4, seed=5, radius=2.0)
    r = oracle.cast_rays(net, o, d, "fixed", delta=1e-3, max_iters=3)
    assert np.all(r["iters"] <= 3)
    assert np.all((r["status"] == 2) | (r["status"] == 1))
