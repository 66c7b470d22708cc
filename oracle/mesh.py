"""Dense marching-tetrahedra mesh of f = 0 on a regular grid (FP64).

TEST INFRASTRUCTURE. Only the tests call this module; the product library
never imports it.

What it computes: the surface that hierarchical mesh extraction (Sec. 4.7)
produces when every cell of the finest grid is meshed, the reference the
leaf-only GPU mesh must reproduce. The grid has 2^n cells per axis over the
root box, f is evaluated at every grid point with the FP64 oracle forward
pass, and every cell is cut into the six tetrahedra that share its main
diagonal (corner bits x = 1, y = 2, z = 4; the tetrahedron of axis order
(a, b, c) runs 0 -> e_a -> e_a + e_b -> 7). In a tetrahedron a corner is
negative when f < 0. One negative (or one non-negative) corner gives one
triangle through the three edges at that corner; two and two give the
quadrilateral through the four crossing edges, split into two triangles. A
crossing point is the linear interpolation of f along the edge, taken from
the endpoint with the lower grid index. Each triangle is oriented so that
its normal has a positive dot product with the gradient of the
tetrahedron's linear interpolant (it faces the f >= 0 side).

Plain numpy, one vectorised pass per tetrahedron type and case; written
from the description above, sharing nothing with the CUDA path.
"""
from __future__ import annotations

import numpy as np

from . import evaluate

# tetrahedra of the cube: axis orders, corners along the path 0 -> 7
_AXIS_ORDERS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def _path(order):
    bits, out = 0, [0]
    for ax in order:
        bits |= 1 << ax
        out.append(bits)
    return out


def grid_values(net, n, lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0)):
    """f at the (2^n + 1)^3 grid points, array [z][y][x], and the axes."""
    R = 1 << n
    axes = [np.asarray(lo[d], np.float64) + (np.asarray(hi[d], np.float64) - lo[d]) *
            (np.arange(R + 1, dtype=np.float64) / R) for d in range(3)]
    zz, yy, xx = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    pts = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1)
    f = evaluate(net, pts).reshape(R + 1, R + 1, R + 1)
    return f, axes


def mesh_dense(net=None, n=4, lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0), values=None, axes=None):
    """Triangles [T, 3, 3] (float64) of the zero set on the 2^n grid. Pass
    values/axes (from grid_values or any function sampled on the grid) to
    skip the network evaluation."""
    if values is None:
        values, axes = grid_values(net, n, lo, hi)
    f = np.asarray(values, np.float64)
    R = f.shape[0] - 1
    h = np.array([axes[d][1] - axes[d][0] for d in range(3)])
    # cell indices of every cube
    cz, cy, cx = np.meshgrid(np.arange(R), np.arange(R), np.arange(R), indexing="ij")
    cx, cy, cz = cx.ravel(), cy.ravel(), cz.ravel()
    out = []
    for t, order in enumerate(_AXIS_ORDERS):
        corners = _path(order)
        gx = [cx + (c & 1) for c in corners]
        gy = [cy + ((c >> 1) & 1) for c in corners]
        gz = [cz + ((c >> 2) & 1) for c in corners]
        fv = np.stack([f[gz[k], gy[k], gx[k]] for k in range(4)], 1)           # [cells, 4]
        pos = np.stack([np.stack([axes[0][gx[k]], axes[1][gy[k]], axes[2][gz[k]]], 1)
                        for k in range(4)], 1)                                   # [cells, 4, 3]
        gid = np.stack([(gz[k] * (R + 1) + gy[k]) * (R + 1) + gx[k] for k in range(4)], 1)
        grad = np.zeros((len(cx), 3))
        for s, ax in enumerate(order):
            grad[:, ax] = (fv[:, s + 1] - fv[:, s]) / h[ax]
        neg = fv < 0.0
        cnt = neg.sum(1)

        def cross(rows, a, b):
            # crossing on edge (a, b) of the given cells, from the lower grid index
            swap = gid[rows, a] > gid[rows, b]
            u = np.where(swap, b, a)
            w = np.where(swap, a, b)
            fu, fw = fv[rows, u], fv[rows, w]
            pu, pw = pos[rows, u], pos[rows, w]
            tt = fu / (fu - fw)
            return pu + tt[:, None] * (pw - pu)

        def orient(v0, v1, v2, g):
            nrm = np.cross(v1 - v0, v2 - v0)
            flip = (nrm * g).sum(1) < 0
            a = np.where(flip[:, None], v2, v1)
            b = np.where(flip[:, None], v1, v2)
            return np.stack([v0, a, b], 1)

        # one corner on its own side
        rows = np.nonzero((cnt == 1) | (cnt == 3))[0]
        if len(rows):
            lone_is_neg = cnt[rows] == 1
            side = neg[rows] == lone_is_neg[:, None]
            lone = np.argmax(side, 1)
            others = np.array([[q for q in range(4) if q != l] for l in range(4)])[lone]
            e = [cross(rows, lone, others[:, j]) for j in range(3)]
            out.append((rows * 6 + t, 0, orient(e[0], e[1], e[2], grad[rows])))
        # two and two: quad (n0,p0) (n0,p1) (n1,p1) (n1,p0)
        rows = np.nonzero(cnt == 2)[0]
        if len(rows):
            order_neg = np.argsort(~neg[rows], 1, kind="stable")  # negatives first, in corner order
            n0, n1, p0, p1 = (order_neg[:, j] for j in range(4))
            e0, e1 = cross(rows, n0, p0), cross(rows, n0, p1)
            e2, e3 = cross(rows, n1, p1), cross(rows, n1, p0)
            out.append((rows * 6 + t, 0, orient(e0, e1, e2, grad[rows])))
            out.append((rows * 6 + t, 1, orient(e0, e2, e3, grad[rows])))
    if not out:
        return np.zeros((0, 3, 3))
    key = np.concatenate([k * 2 + j for k, j, _ in out])
    tris = np.concatenate([tr for _, _, tr in out])
    return tris[np.argsort(key, kind="stable")]


def edges(tris, decimals=12):
    """Undirected edges with multiplicity, from vertices rounded for matching:
    dict {(vertex a, vertex b): [count of a->b, count of b->a]}."""
    vs = np.round(tris, decimals)
    out = {}
    for tri in vs:
        for a, b in ((0, 1), (1, 2), (2, 0)):
            p, q = tuple(tri[a]), tuple(tri[b])
            k = (p, q) if p < q else (q, p)
            d = out.setdefault(k, [0, 0])
            d[0 if p < q else 1] += 1
    return out


def euler_characteristic(tris, decimals=12):
    """V - E + F of the triangle soup with vertices merged by position."""
    vs = np.round(tris.reshape(-1, 3), decimals)
    V = len({tuple(v) for v in vs})
    E = len(edges(tris, decimals))
    return V - E + len(tris)


def signed_volume(tris):
    """Sum of v0 . (v1 x v2) / 6: the enclosed volume for a closed surface
    whose triangles face outward."""
    return float(np.einsum("ij,ij->i", tris[:, 0], np.cross(tris[:, 1], tris[:, 2])).sum() / 6.0)


def area(tris):
    return float(0.5 * np.linalg.norm(np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0]), axis=1).sum())

