"""Pins of the dense marching-tetrahedra oracle (oracle/mesh.py) against
closed forms and topology: planes are reproduced exactly, closed surfaces
are watertight with the right Euler characteristic and enclose the right
volume with outward-facing triangles."""
import math

import numpy as np
import pytest

import oracle
from oracle import mesh as om
from paper_2202_02444_gb300 import workloads as wl


def sampled(fn, n, lo=-1.0, hi=1.0):
    R = 1 << n
    ax = lo + (hi - lo) * np.arange(R + 1, dtype=np.float64) / R
    zz, yy, xx = np.meshgrid(ax, ax, ax, indexing="ij")
    return fn(xx, yy, zz), [ax, ax, ax]


def test_plane_is_exact():
    nv = np.array([0.2, 0.1, 1.0])
    d = 0.137
    f, axes = sampled(lambda x, y, z: nv[0] * x + nv[1] * y + nv[2] * z - d, 4)
    tris = om.mesh_dense(values=f, axes=axes)
    assert len(tris) > 0
    # every vertex on the plane (linear interpolation of a linear function)
    assert np.abs(tris @ nv - d).max() < 1e-12
    # triangles face the f >= 0 side: along +n
    nrm = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    assert (nrm @ nv > 0).all()
    # the plane crosses every vertical line of the box: area = 4 |n| / n_z
    assert om.area(tris) == pytest.approx(4.0 * np.linalg.norm(nv) / nv[2], rel=1e-12)


def test_plane_net_through_the_oracle_forward_pass():
    nv = np.array([0.3, -0.5, 0.8])
    mlp = wl.make_custom_mlp([3, 1], [], [(nv[None, :], np.array([-0.1]))])
    tris = om.mesh_dense(mlp, n=3)
    n32 = nv.astype(np.float32).astype(np.float64)
    b32 = float(np.float32(-0.1))
    assert np.abs(tris @ n32 + b32).max() < 1e-9
    nrm = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    assert (nrm @ n32 > 0).all()


def test_sphere_closed_and_measured():
    r = 0.6
    f, axes = sampled(lambda x, y, z: np.sqrt(x * x + y * y + z * z) - r, 5)
    tris = om.mesh_dense(values=f, axes=axes)
    e = om.edges(tris)
    # watertight and consistently oriented: every edge once in each direction
    assert all(c == [1, 1] for c in e.values())
    assert om.euler_characteristic(tris) == 2
    assert om.signed_volume(tris) == pytest.approx(4 / 3 * math.pi * r ** 3, rel=0.02)
    assert om.area(tris) == pytest.approx(4 * math.pi * r ** 2, rel=0.02)
    v = tris.reshape(-1, 3)
    assert np.abs(np.linalg.norm(v, axis=1) - r).max() < (2 / 32) ** 2


def test_torus_has_euler_characteristic_zero():
    R, r = 0.55, 0.22
    f, axes = sampled(lambda x, y, z: (np.sqrt(x * x + y * y) - R) ** 2 + z * z - r * r, 5)
    tris = om.mesh_dense(values=f, axes=axes)
    assert all(c == [1, 1] for c in om.edges(tris).values())
    assert om.euler_characteristic(tris) == 0
    assert om.signed_volume(tris) == pytest.approx(2 * math.pi ** 2 * R * r * r, rel=0.05)


def cube_net(r):
    """ReLU net of f = max(|x|, |y|, |z|) - r: |t| = relu(t) + relu(-t),
    max(a, b) = a + relu(b - a) (a >= 0)."""
    W1 = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    W2 = np.array([[1, 1, 0, 0, 0, 0], [-1, -1, 1, 1, 0, 0], [0, 0, 0, 0, 1, 1]], float)
    W3 = np.array([[1, 1, 0], [-1, -1, 1]], float)
    W4 = np.array([[1, 1]], float)
    return wl.make_custom_mlp([3, 6, 3, 2, 1], [1, 1, 1],
                              [(W1, np.zeros(6)), (W2, np.zeros(3)), (W3, np.zeros(2)), (W4, np.array([-r]))])


def test_cube_net_closed_outward():
    r = 0.53
    mlp = cube_net(r)
    x = np.random.default_rng(0).uniform(-1, 1, (200, 3))
    assert np.allclose(oracle.evaluate(mlp, x), np.abs(x).max(1) - np.float32(r), atol=1e-6)
    tris = om.mesh_dense(mlp, n=4)
    assert all(c == [1, 1] for c in om.edges(tris).values())
    assert om.euler_characteristic(tris) == 2
    vol = om.signed_volume(tris)
    assert 0 < vol <= (2 * r) ** 3 + 1e-9
    assert vol == pytest.approx((2 * r) ** 3, rel=0.05)


def test_no_sign_change_no_triangles():
    f, axes = sampled(lambda x, y, z: x * x + y * y + z * z + 0.1, 3)
    assert len(om.mesh_dense(values=f, axes=axes)) == 0
