"""GPU mesh of the zero set inside octree leaves (sra_mesh_leaves) against the
dense FP64 marching-tetrahedra oracle, and the hierarchical property: the
mesh of the UNKNOWN leaves alone equals the mesh of every cell."""
import numpy as np
import pytest
import torch

from oracle import mesh as om
from paper_2202_02444_gb300 import workloads as wl

from test_oracle_mesh import cube_net

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sra():
    from paper_2202_02444_gb300 import sra as s
    return s


def all_cells(level):
    m = 1 << level
    iz, iy, ix = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    nodes = np.zeros(m ** 3, wl.NODE_DTYPE)
    nodes["ix"], nodes["iy"], nodes["iz"], nodes["level"] = ix.ravel(), iy.ravel(), iz.ravel(), level
    return nodes


def sorted_rows(t):
    a = t.reshape(len(t), 9)
    return a[np.lexsort(a.T[::-1])]


def match_sets(got, ref, tol):
    """Every GPU triangle has an oracle triangle within tol (vertex-wise) and
    the counts agree."""
    from scipy.spatial import cKDTree
    assert len(got) == len(ref), (len(got), len(ref))
    tree = cKDTree(ref.reshape(len(ref), 9))
    d, _ = tree.query(got.reshape(len(got), 9).astype(np.float64))
    assert d.max() < tol, d.max()


def test_dense_grid_matches_oracle(sra):
    mlp = wl.net_small_relu()
    level, sub = 3, 2
    net = sra.Net(mlp)
    try:
        leaves = sra.nodes_to_tensor(all_cells(level))
        tris = sra.mesh_leaves(net, leaves, sub).cpu().numpy()
    finally:
        net.close()
    f, axes = om.grid_values(mlp, level + sub)
    assert np.abs(f).min() > 1e-6  # no grid value close enough to zero to flip a sign in FP32 (error ~1e-7)
    ref = om.mesh_dense(values=f, axes=axes)
    match_sets(tris, ref, 1e-5)


def test_leaves_only_equals_every_cell(sra):
    """Cells that range analysis proves POSITIVE or NEGATIVE hold no surface:
    meshing only the UNKNOWN leaves gives the same triangles, bit for bit."""
    mlp = wl.make_mlp([64, 64], "elu", seed=90)
    level, sub = 4, 3
    net = sra.Net(mlp)
    try:
        leaves, counts = sra.extract_leaves(net, level, opts=sra.make_opts(arith="truncate", K=16))
        assert 0 < leaves.shape[0] < 8 ** level
        a = sra.mesh_leaves(net, leaves, sub).cpu().numpy()
        b = sra.mesh_leaves(net, sra.nodes_to_tensor(all_cells(level)), sub).cpu().numpy()
    finally:
        net.close()
    assert len(a) > 0
    assert np.array_equal(sorted_rows(a), sorted_rows(b))


def test_cube_net_closed_surface(sra):
    r = 0.53
    mlp = cube_net(r)
    net = sra.Net(mlp)
    try:
        leaves, _ = sra.extract_leaves(net, 3, opts=sra.make_opts(arith="fixed"))
        tris = sra.mesh_leaves(net, leaves, 2).cpu().numpy().astype(np.float64)
    finally:
        net.close()
    assert all(c == [1, 1] for c in om.edges(tris).values())
    assert om.euler_characteristic(tris) == 2
    assert om.signed_volume(tris) == pytest.approx((2 * r) ** 3, rel=0.05)
    ref = om.mesh_dense(mlp, n=5)
    assert len(tris) == len(ref)


def test_capacity_and_arguments(sra):
    mlp = wl.net_small_relu()
    net = sra.Net(mlp)
    try:
        leaves = sra.nodes_to_tensor(all_cells(2))
        full = sra.mesh_leaves(net, leaves, 2)
        small = sra.mesh_leaves(net, leaves, 2, cap=5)  # retries with the reported count
        assert torch.equal(full, small)
        with pytest.raises(sra.SraError) as e:
            sra.mesh_leaves(net, leaves, 6)
        assert e.value.code == sra.EINVAL
        assert sra.mesh_leaves(net, leaves[:0], 3).shape[0] == 0
    finally:
        net.close()
