"""Pins of the convergence test of Proc. 3 in the oracle tree builder: the
fixed-depth tree when no node is small enough, leaves within delta of an
analytic plane, and every converged leaf small with a sign change across its
face centres."""
import math

import numpy as np

import oracle
from paper_2202_02444_gb300 import workloads as wl

XL, XU = (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)


def boxes(nodes):
    w = 2.0 / (1 << nodes["level"].astype(np.int64))
    lo = -1.0 + np.stack([nodes["ix"], nodes["iy"], nodes["iz"]], 1) * w[:, None]
    return lo, lo + w[:, None], w


def test_no_small_node_gives_the_fixed_depth_tree():
    mlp = wl.net_small_relu()
    a, ca = oracle.build_tree(mlp, XL, XU, 5)
    b, cb = oracle.build_tree(mlp, XL, XU, 5, delta=1e-3)  # level-5 cells are 1/16 wide
    assert np.array_equal(a, b) and cb[4] == 0 and np.array_equal(ca, cb[:4])


def test_plane_leaves_within_delta():
    nv = np.array([0.3, -0.5, 0.8])
    d = 0.1
    mlp = wl.make_custom_mlp([3, 1], [], [(nv[None, :], np.array([-d]))])
    delta = 0.2
    nodes, cnt = oracle.build_tree(mlp, XL, XU, 9, delta=delta)
    unk = nodes[nodes["cls"] == oracle.UNKNOWN]
    lo, hi, w = boxes(unk)
    n32 = nv.astype(np.float32).astype(np.float64)
    d32 = float(np.float32(d))
    c = 0.5 * (lo + hi)
    dist = np.abs(c @ n32 - d32) / np.linalg.norm(n32)
    # affine bounds of a linear function are exact: every UNKNOWN leaf meets the plane
    assert (dist <= 0.5 * math.sqrt(3) * w + 1e-12).all()
    # leaves above the depth cap were stopped by the convergence test: small,
    # and every point of them within delta of the plane
    early = unk["level"] < 9
    assert 0 < early.sum() <= cnt[4]
    assert (w[early] < delta / math.sqrt(3)).all()
    assert (dist[early] + 0.5 * math.sqrt(3) * w[early] <= delta).all()
    # a small box the plane crosses near a corner keeps all face centres on one
    # side; the test does not stop it, so it continues to the depth cap
    assert (~early).sum() > 0


def test_converged_leaves_change_sign_on_faces():
    mlp = wl.make_mlp([32, 32], "elu", seed=3)
    delta = 0.05
    nodes, cnt = oracle.build_tree(mlp, XL, XU, 8, delta=delta)
    unk = nodes[nodes["cls"] == oracle.UNKNOWN]
    lo, hi, w = boxes(unk)
    small = w < delta / math.sqrt(3)
    conv = 0
    for i in np.nonzero(small)[0]:
        c = 0.5 * (lo[i] + hi[i])
        pts = np.repeat(c[None], 6, 0)
        for f in range(6):
            pts[f, f >> 1] = hi[i, f >> 1] if f & 1 else lo[i, f >> 1]
        v = oracle.evaluate(mlp, pts)
        if unk["level"][i] < 8:  # above the depth cap only the convergence test stops a node
            assert (v < 0).any() and (v > 0).any()
        conv += bool((v < 0).any() and (v > 0).any())
    assert conv == cnt[4] > 0
