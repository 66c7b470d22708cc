"""Python wrapper over the FP64 C oracle (``sra_oracle.c``).

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / reference leg call this module. The product
library never imports it.

The C library is compiled on first use (or by ``build()``) with plain gcc,
no fast-math and no floating-point contraction, so x86-64 and aarch64 hosts
produce the same doubles.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sra_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

INTERVAL, AFFINE_FIXED, AFFINE_TRUNCATE, AFFINE_FULL = 0, 1, 2, 3
CHEBYSHEV, MINRANGE = 0, 1
UNKNOWN, POSITIVE, NEGATIVE = 0, 1, 2
OCTREE, KD = 0, 1
ARITH = {"interval": INTERVAL, "fixed": AFFINE_FIXED, "truncate": AFFINE_TRUNCATE,
         "full": AFFINE_FULL}
SLOPE = {"chebyshev": CHEBYSHEV, "minrange": MINRANGE}


def build(force=False):
    """Compile liboracle.so next to the source if missing or stale."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                   "-ffp-contract=off", "-fno-fast-math", "-D_GNU_SOURCE",
                   "-o", tmp, _SRC, "-lm"]
            subprocess.check_call(cmd, cwd=_HERE)
            os.replace(tmp, _LIB)
    return _LIB


class _Net(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("widths", C.POINTER(C.c_int)),
                ("acts", C.POINTER(C.c_int)), ("params", C.POINTER(C.c_double)),
                ("pe_octaves", C.c_int)]


class _Opts(C.Structure):
    _fields_ = [("arith", C.c_int), ("K", C.c_int), ("slope", C.c_int)]


class _RayOpts(C.Structure):
    _fields_ = [("delta", C.c_double), ("t_max", C.c_double), ("sigma0", C.c_double),
                ("eta_plus", C.c_double), ("eta_minus", C.c_double),
                ("safety", C.c_double), ("max_iters", C.c_int64)]


NODE_CDT = np.dtype([("ix", "<u2"), ("iy", "<u2"), ("iz", "<u2"), ("level", "<u2"),
                     ("cls", "<i4")])


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        L.orc_linearize.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, dp, dp, dp]
        L.orc_interval_act.argtypes = [C.c_int, C.c_double, C.c_double, dp, dp]
        L.orc_eval.restype = C.c_double
        L.orc_eval.argtypes = [C.POINTER(_Net), dp]
        L.orc_eval_batch.argtypes = [C.POINTER(_Net), C.c_int64, dp, dp, C.c_int]
        L.orc_range_bound.restype = C.c_int
        L.orc_range_bound.argtypes = [C.POINTER(_Net), C.POINTER(_Opts), dp, dp, C.c_int,
                                      dp, dp, dp, dp]
        L.orc_bound_boxes.argtypes = [C.POINTER(_Net), C.POINTER(_Opts), C.c_int64, dp, dp,
                                      dp, dp, dp, dp, C.POINTER(C.c_int32), dp, C.c_int]
        L.orc_build_tree.restype = C.c_int64
        L.orc_build_tree.argtypes = [C.POINTER(_Net), C.POINTER(_Opts), dp, dp, C.c_int,
                                     C.c_int, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]
        L.orc_build_tree_conv.restype = C.c_int64
        L.orc_build_tree_conv.argtypes = [C.POINTER(_Net), C.POINTER(_Opts), dp, dp, C.c_int,
                                          C.c_int, C.c_double, C.c_void_p, C.c_int64,
                                          C.POINTER(C.c_int64)]
        L.orc_classify_nodes.argtypes = [C.POINTER(_Net), C.POINTER(_Opts), dp, dp, C.c_int,
                                         C.c_int64, C.c_void_p, C.POINTER(C.c_int32), dp, dp,
                                         dp, C.c_int]
        L.orc_cast_ray.restype = C.c_int
        L.orc_cast_rays.argtypes = [C.POINTER(_Net), C.POINTER(_Opts), C.POINTER(_RayOpts),
                                    C.c_int64, dp, dp, dp, C.POINTER(C.c_int64),
                                    C.POINTER(C.c_int32), dp, C.c_int]
        L.orc_max_threads.restype = C.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class OracleNet:
    """Holds the FP64 copy of an MLP (the float32 parameters widened exactly)."""

    def __init__(self, mlp):
        self.mlp = mlp
        self._w = np.ascontiguousarray(mlp.widths, dtype=np.int32)
        self._a = np.ascontiguousarray(mlp.acts if len(mlp.acts) else [0], dtype=np.int32)
        self._p = np.ascontiguousarray(mlp.params, dtype=np.float64)
        self.s = _Net(mlp.n_layers, self._w.ctypes.data_as(C.POINTER(C.c_int)),
                      self._a.ctypes.data_as(C.POINTER(C.c_int)), _dp(self._p),
                      int(mlp.pe_octaves))


def _net(net):
    return net if isinstance(net, OracleNet) else OracleNet(net)


def _opts(arith="fixed", K=0, slope="chebyshev"):
    a = ARITH[arith] if isinstance(arith, str) else int(arith)
    s = SLOPE[slope] if isinstance(slope, str) else int(slope)
    return _Opts(a, int(K), s)


def max_threads():
    return lib().orc_max_threads()


def linearize(act, l, u, slope="chebyshev"):
    a, b, g = C.c_double(), C.c_double(), C.c_double()
    s = SLOPE[slope] if isinstance(slope, str) else int(slope)
    lib().orc_linearize(int(act), s, float(l), float(u), C.byref(a), C.byref(b), C.byref(g))
    return a.value, b.value, g.value


def interval_act(act, l, u):
    lo, hi = C.c_double(), C.c_double()
    lib().orc_interval_act(int(act), float(l), float(u), C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def evaluate(net, x, nthreads=0):
    """Plain forward pass f(x) for x of shape (n, 3)."""
    n = _net(net)
    x = np.ascontiguousarray(np.asarray(x, np.float64).reshape(-1, 3))
    out = np.empty(len(x), np.float64)
    lib().orc_eval_batch(C.byref(n.s), len(x), _dp(x), _dp(out), int(nthreads))
    return out


def range_bound(net, center, axes, arith="fixed", K=0, slope="chebyshev"):
    """Proc. 1 on one box: returns (cls, lo, hi, y0, rad)."""
    n = _net(net)
    o = _opts(arith, K, slope)
    c = np.ascontiguousarray(np.asarray(center, np.float64).reshape(3))
    ax = np.ascontiguousarray(np.asarray(axes, np.float64).reshape(-1, 3))
    lo, hi, y0, rad = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    cls = lib().orc_range_bound(C.byref(n.s), C.byref(o), _dp(c), _dp(ax), len(ax),
                                C.byref(lo), C.byref(hi), C.byref(y0), C.byref(rad))
    return cls, lo.value, hi.value, y0.value, rad.value


def bound_boxes(net, centers, halfw, arith="fixed", K=0, slope="chebyshev", nthreads=0):
    """Proc. 1 on axis-aligned boxes: returns dict of lo, hi, y0, rad, cls."""
    n = _net(net)
    o = _opts(arith, K, slope)
    c = np.ascontiguousarray(np.asarray(centers, np.float64).reshape(-1, 3))
    h = np.ascontiguousarray(np.asarray(halfw, np.float64).reshape(-1, 3))
    m = len(c)
    lo, hi, y0, rad, gap = (np.empty(m) for _ in range(5))
    cls = np.empty(m, np.int32)
    lib().orc_bound_boxes(C.byref(n.s), C.byref(o), m, _dp(c), _dp(h), _dp(lo), _dp(hi),
                          _dp(y0), _dp(rad), cls.ctypes.data_as(C.POINTER(C.c_int32)),
                          _dp(gap), int(nthreads))
    return {"lo": lo, "hi": hi, "y0": y0, "rad": rad, "cls": cls, "sel_gap": gap}


def build_tree(net, xl, xu, max_level, split=OCTREE, arith="fixed", K=0,
               slope="chebyshev", cap=1 << 22, delta=None):
    """Proc. 3: (nodes with cls, counts[pos, neg, unk, calls(, converged)]).
    Fixed depth; with delta, also the convergence test for small nodes."""
    n = _net(net)
    o = _opts(arith, K, slope)
    xl = np.ascontiguousarray(np.asarray(xl, np.float64).reshape(3))
    xu = np.ascontiguousarray(np.asarray(xu, np.float64).reshape(3))
    out = np.zeros(cap, NODE_CDT)
    if delta is None:
        counts = (C.c_int64 * 4)()
        m = lib().orc_build_tree(C.byref(n.s), C.byref(o), _dp(xl), _dp(xu), int(max_level),
                                 int(split), out.ctypes.data, cap, counts)
    else:
        counts = (C.c_int64 * 5)()
        m = lib().orc_build_tree_conv(C.byref(n.s), C.byref(o), _dp(xl), _dp(xu), int(max_level),
                                      int(split), float(delta), out.ctypes.data, cap, counts)
    if m > cap:
        return build_tree(net, xl, xu, max_level, split, arith, K, slope, cap=int(m), delta=delta)
    return out[:m].copy(), np.array(list(counts), np.int64)


def classify_nodes(net, nodes, xl, xu, split=OCTREE, arith="fixed", K=0,
                   slope="chebyshev", nthreads=0):
    """RangeBound on a list of tree nodes: returns (cls, lo, hi)."""
    n = _net(net)
    o = _opts(arith, K, slope)
    xl = np.ascontiguousarray(np.asarray(xl, np.float64).reshape(3))
    xu = np.ascontiguousarray(np.asarray(xu, np.float64).reshape(3))
    nd = np.zeros(len(nodes), NODE_CDT)
    for f in ("ix", "iy", "iz", "level"):
        nd[f] = nodes[f]
    cls = np.empty(len(nodes), np.int32)
    lo = np.empty(len(nodes))
    hi = np.empty(len(nodes))
    gap = np.empty(len(nodes))
    lib().orc_classify_nodes(C.byref(n.s), C.byref(o), _dp(xl), _dp(xu), int(split),
                             len(nodes), nd.ctypes.data,
                             cls.ctypes.data_as(C.POINTER(C.c_int32)), _dp(lo), _dp(hi),
                             _dp(gap), int(nthreads))
    return cls, lo, hi, gap


def cast_rays(net, origins, dirs, arith="fixed", K=0, slope="chebyshev", delta=1e-3,
              t_max=10.0, sigma0=None, eta_plus=1.5, eta_minus=0.5, safety=0.98,
              max_iters=1 << 20, nthreads=0):
    """Proc. 2 per ray: returns dict t (inf = miss), iters, status, margin."""
    n = _net(net)
    o = _opts(arith, K, slope)
    if sigma0 is None:
        sigma0 = t_max / 10.0
    ro = _RayOpts(delta, t_max, sigma0, eta_plus, eta_minus, safety, int(max_iters))
    p = np.ascontiguousarray(np.asarray(origins, np.float64).reshape(-1, 3))
    r = np.ascontiguousarray(np.asarray(dirs, np.float64).reshape(-1, 3))
    m = len(p)
    t = np.empty(m)
    it = np.empty(m, np.int64)
    st = np.empty(m, np.int32)
    mg = np.empty(m)
    lib().orc_cast_rays(C.byref(n.s), C.byref(o), C.byref(ro), m, _dp(p), _dp(r), _dp(t),
                        it.ctypes.data_as(C.POINTER(C.c_int64)),
                        st.ctypes.data_as(C.POINTER(C.c_int32)), _dp(mg), int(nthreads))
    return {"t": t, "iters": it, "status": st, "margin": mg}


def empty_spheres(net, points, r_max, levels, arith="fixed", K=0, slope="chebyshev"):
    """Empty-sphere query (Sec. 4.4): for each point p, the largest
    r = r_max * 2^-k (0 <= k < levels) such that RangeBound (Proc. 1) of the
    box [p - r, p + r] is POSITIVE or NEGATIVE, else 0. The box contains the
    ball of radius r around p, which therefore misses the zero set."""
    points = np.asarray(points, np.float64).reshape(-1, 3)
    radius = np.zeros(len(points))
    open_ = np.arange(len(points))
    r = float(r_max)
    for _ in range(int(levels)):
        if len(open_) == 0:
            break
        res = bound_boxes(net, points[open_], np.full((len(open_), 3), r), arith, K, slope)
        done = res["cls"] != UNKNOWN
        radius[open_[done]] = r
        open_ = open_[~done]
        r *= 0.5
    return radius
