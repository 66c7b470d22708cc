"""Python binding of libsra.so (ctypes; argument marshalling only).

Every function takes CUDA torch tensors, passes their device pointers and the
current torch stream to the C ABI declared in include/sra.h, and returns
tensors. All compute runs in the library's CUDA kernels; there is no CPU or
PyTorch fallback: importing this module fails if libsra.so is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsra.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
_lib = C.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ECAPACITY, EUNSUPPORTED = range(7)
UNKNOWN, POSITIVE, NEGATIVE = 0, 1, 2
ARITH = {"interval": 0, "fixed": 1, "truncate": 2, "full": 3}
SLOPE = {"chebyshev": 0, "minrange": 1}
PRECISION = {"fp32": 0, "fp64": 1, "bf16_sound": 2, "bf16": 3}
SPLIT = {"octree": 0, "kd": 1}
CNT_CHILDREN, CNT_LEAVES, CNT_POSITIVE, CNT_NEGATIVE, CNT_UNKNOWN, CNT_RECHECKED, CNT_CONVERGED = range(7)
CNT_N = 8

NODE_DTYPE = np.dtype([("ix", "<u2"), ("iy", "<u2"), ("iz", "<u2"), ("level", "<u2")])


class SraError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sra error {code}: {msg}")
        self.code = code


class MlpDesc(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("widths", C.POINTER(C.c_int32)),
                ("acts", C.POINTER(C.c_int32)), ("params", C.POINTER(C.c_float)),
                ("pe_octaves", C.c_int32)]


class Opts(C.Structure):
    _fields_ = [("arith", C.c_int32), ("K", C.c_int32), ("slope", C.c_int32),
                ("precision", C.c_int32), ("recheck", C.c_int32), ("recheck_band", C.c_float),
                ("split", C.c_int32), ("delta", C.c_float), ("t_max", C.c_float),
                ("sigma0", C.c_float), ("eta_plus", C.c_float), ("eta_minus", C.c_float),
                ("safety", C.c_float), ("max_iters", C.c_int64),
                ("block_threads", C.c_int32), ("converge", C.c_int32),
                ("recheck_count", C.c_void_p)]


class Request(C.Structure):
    """One query of a serving trace (sra_request)."""
    _fields_ = [("kind", C.c_int32), ("net", C.c_int32), ("form", C.c_int32), ("depth", C.c_int32),
                ("arrival", C.c_double), ("n", C.c_int64),
                ("a", C.c_void_p), ("b", C.c_void_p), ("lo", C.c_void_p), ("hi", C.c_void_p),
                ("iters", C.c_void_p), ("cls", C.c_void_p), ("leaves", C.c_void_p),
                ("cap", C.c_int64), ("n_out", C.c_int64), ("status", C.c_int32),
                ("slot", C.c_int32), ("levels", C.c_int32), ("pad", C.c_int32),
                ("t_admit", C.c_double), ("t_done", C.c_double)]


class ServeCfg(C.Structure):
    _fields_ = [("slots", C.c_int32), ("realtime", C.c_int32), ("frontier_bytes", C.c_int64)]


REQ_RAYS, REQ_BOXES, REQ_LEAVES = 0, 1, 2


class BatchSeg(C.Structure):
    """One network's frontier in a batched round (sra_batch_seg)."""
    _fields_ = [("net", C.c_int32), ("max_level", C.c_int32), ("first", C.c_int64), ("n", C.c_int64),
                ("out_first", C.c_int64), ("cap_out", C.c_int64), ("leaf_first", C.c_int64),
                ("cap_leaves", C.c_int64)]

_vp = C.c_void_p
_lib.sra_last_error.restype = C.c_char_p
_lib.sra_default_opts.argtypes = [C.POINTER(Opts)]
_lib.sra_load_mlp.argtypes = [C.POINTER(MlpDesc), C.POINTER(_vp)]
_lib.sra_free_mlp.argtypes = [_vp]
_lib.sra_bound_boxes.argtypes = [_vp, C.POINTER(Opts), _vp, _vp, C.c_int64, _vp, _vp, _vp, _vp]
_lib.sra_classify_and_split.argtypes = [_vp, C.POINTER(Opts), C.POINTER(C.c_float),
                                        C.POINTER(C.c_float), _vp, C.c_int64, C.c_int32, _vp,
                                        C.c_int64, _vp, C.c_int64, _vp, _vp]
_lib.sra_cast_rays.argtypes = [_vp, C.POINTER(Opts), _vp, _vp, C.c_int64, _vp, _vp, _vp]
_lib.sra_extract_leaves.argtypes = [_vp, C.POINTER(Opts), C.POINTER(C.c_float),
                                    C.POINTER(C.c_float), C.c_int32, _vp, C.c_int64,
                                    C.POINTER(C.c_int64), C.POINTER(C.c_int64), _vp]
_lib.sra_eval.argtypes = [_vp, _vp, C.c_int64, _vp, _vp]
_lib.sra_sync_status.argtypes = [_vp, _vp]
_lib.sra_classify_and_split_batch.argtypes = [C.POINTER(_vp), C.POINTER(Opts), C.c_int32,
                                              C.POINTER(C.c_float), C.POINTER(C.c_float), _vp,
                                              C.POINTER(BatchSeg), C.c_int32, _vp, _vp, _vp, _vp]
_lib.sra_mesh_leaves.argtypes = [_vp, C.POINTER(C.c_float), C.POINTER(C.c_float), _vp, C.c_int64, C.c_int32,
                                 _vp, C.c_int64, C.POINTER(C.c_int64), _vp]
_lib.sra_empty_spheres.argtypes = [_vp, C.POINTER(Opts), _vp, C.c_int64, C.c_float, C.c_int32, _vp, _vp]
_lib.sra_cast_frustum.argtypes = [_vp, C.POINTER(Opts), C.POINTER(C.c_float), _vp, C.c_int32, C.c_int32,
                                  C.c_int32, _vp, _vp, C.POINTER(C.c_int64), _vp]
_lib.sra_serve.argtypes = [C.POINTER(_vp), C.c_int32, C.POINTER(Opts), C.c_int32,
                           C.POINTER(ServeCfg), C.POINTER(Request), C.c_int64]
for _f in ("sra_load_mlp", "sra_free_mlp", "sra_bound_boxes", "sra_classify_and_split",
           "sra_cast_rays", "sra_extract_leaves", "sra_eval", "sra_sync_status", "sra_serve",
           "sra_classify_and_split_batch", "sra_mesh_leaves", "sra_empty_spheres", "sra_cast_frustum"):
    getattr(_lib, _f).restype = C.c_int


def library():
    """The loaded ctypes library (for tests that call the ABI directly)."""
    return _lib


def _check(code):
    if code != OK:
        raise SraError(code, _lib.sra_last_error().decode())


def make_opts(arith="fixed", K=0, slope="chebyshev", precision="fp32", recheck=False,
              recheck_band=1e-5, split="octree", delta=None, t_max=None, sigma0=None,
              eta_plus=None, eta_minus=None, safety=None, max_iters=None, block_threads=0,
              converge=False, recheck_count=None):
    """sra_opts; recheck_count is an optional CUDA int64 tensor that the FP64
    re-check adds its box / ray count to (the caller keeps it alive)."""
    o = Opts()
    _lib.sra_default_opts(C.byref(o))
    o.arith = ARITH[arith] if isinstance(arith, str) else int(arith)
    o.K = int(K)
    o.slope = SLOPE[slope] if isinstance(slope, str) else int(slope)
    o.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    o.recheck = int(bool(recheck))
    o.recheck_band = float(recheck_band)
    o.split = SPLIT[split] if isinstance(split, str) else int(split)
    for k, v in (("delta", delta), ("t_max", t_max), ("sigma0", sigma0), ("eta_plus", eta_plus),
                 ("eta_minus", eta_minus), ("safety", safety)):
        if v is not None:
            setattr(o, k, float(v))
    if t_max is not None and sigma0 is None:
        o.sigma0 = float(t_max) / 10.0
    if max_iters is not None:
        o.max_iters = int(max_iters)
    o.block_threads = int(block_threads)
    o.converge = int(bool(converge))
    if recheck_count is not None:
        _need_count(recheck_count)
        o.recheck_count = recheck_count.data_ptr()
    return o


def _need_count(t):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.int64 and t.numel() >= 1
            and t.is_contiguous()):
        raise ValueError("recheck_count must be a contiguous CUDA int64 tensor")


def _stream():
    return _vp(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return _vp(t.data_ptr()) if t is not None else _vp(0)


def sync_status(net):
    """Synchronise the current stream and raise if a tensor-core kernel of
    this net reported a bounded wait that ran out (sra_sync_status)."""
    _check(_lib.sra_sync_status(net.handle, _stream()))


def _need(t, dtype, shape_last=None, name="tensor"):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    if shape_last is not None and t.shape[-1] != shape_last:
        raise ValueError(f"{name} must have last dimension {shape_last}")
    return t


class Net:
    """A network resident on the current device (sra_load_mlp)."""

    def __init__(self, mlp):
        self.mlp = mlp
        w = np.ascontiguousarray(mlp.widths, np.int32)
        a = np.ascontiguousarray(mlp.acts if len(mlp.acts) else [0], np.int32)
        p = np.ascontiguousarray(mlp.params, np.float32)
        d = MlpDesc(mlp.n_layers, w.ctypes.data_as(C.POINTER(C.c_int32)),
                    a.ctypes.data_as(C.POINTER(C.c_int32)),
                    p.ctypes.data_as(C.POINTER(C.c_float)), int(mlp.pe_octaves))
        h = _vp()
        _check(_lib.sra_load_mlp(C.byref(d), C.byref(h)))
        self.handle = h

    def close(self):
        if self.handle:
            _lib.sra_free_mlp(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bound_boxes(net, centers, halfw, opts=None, lo=None, hi=None, cls=None, **kw):
    """Proc. 1 on boxes centers +- halfw (CUDA float32 [n,3]); returns (lo, hi, cls)."""
    opts = opts or make_opts(**kw)
    _need(centers, torch.float32, 3, "centers")
    _need(halfw, torch.float32, 3, "halfw")
    n = centers.shape[0]
    dev = centers.device
    lo = lo if lo is not None else torch.empty(n, dtype=torch.float32, device=dev)
    hi = hi if hi is not None else torch.empty(n, dtype=torch.float32, device=dev)
    cls = cls if cls is not None else torch.empty(n, dtype=torch.uint8, device=dev)
    _check(_lib.sra_bound_boxes(net.handle, C.byref(opts), _ptr(centers), _ptr(halfw), n,
                                _ptr(lo), _ptr(hi), _ptr(cls), _stream()))
    return lo, hi, cls


def evaluate(net, x, out=None):
    """Plain forward pass f(x) for CUDA float32 [n,3]."""
    _need(x, torch.float32, 3, "x")
    out = out if out is not None else torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    _check(_lib.sra_eval(net.handle, _ptr(x), x.shape[0], _ptr(out), _stream()))
    return out


def nodes_to_tensor(nodes, device="cuda"):
    """numpy NODE_DTYPE records -> CUDA int16 tensor [n,4] (the sra_node layout)."""
    a = np.ascontiguousarray(nodes).view(np.int16).reshape(-1, 4)
    return torch.from_numpy(a.copy()).to(device)


def tensor_to_nodes(t):
    a = t.detach().cpu().numpy().astype(np.int16).reshape(-1)
    return a.view(NODE_DTYPE).copy()


def classify_and_split(net, frontier, max_level, root_lo=(-1.0, -1.0, -1.0),
                       root_hi=(1.0, 1.0, 1.0), opts=None, out=None, cap_out=None, leaves=None,
                       cap_leaves=None, counts=None, **kw):
    """One round of Proc. 3; frontier is a CUDA int16 [n,4] node tensor.
    Returns (children, leaves, counts) with counts a CUDA int64[8] tensor."""
    opts = opts or make_opts(**kw)
    _need(frontier, torch.int16, 4, "frontier")
    n = frontier.shape[0]
    dev = frontier.device
    fan = 8 if opts.split == 0 else 2
    if out is None:
        cap_out = n * fan if cap_out is None else cap_out
        out = torch.empty((max(cap_out, 1), 4), dtype=torch.int16, device=dev)
    if leaves is None:
        cap_leaves = n if cap_leaves is None else cap_leaves
        leaves = torch.empty((max(cap_leaves, 1), 4), dtype=torch.int16, device=dev)
    cap_out = out.shape[0] if cap_out is None else cap_out
    cap_leaves = leaves.shape[0] if cap_leaves is None else cap_leaves
    if counts is None:
        counts = torch.zeros(CNT_N, dtype=torch.int64, device=dev)
    rl = (C.c_float * 3)(*root_lo)
    rh = (C.c_float * 3)(*root_hi)
    _check(_lib.sra_classify_and_split(net.handle, C.byref(opts), rl, rh, _ptr(frontier), n,
                                       int(max_level), _ptr(out), int(cap_out), _ptr(leaves),
                                       int(cap_leaves), _ptr(counts), _stream()))
    return out, leaves, counts


def classify_and_split_batch(nets, opts, frontier, segs, out, leaves, counts=None,
                             root_lo=(-1.0, -1.0, -1.0), root_hi=(1.0, 1.0, 1.0)):
    """One round of Proc. 3 over many networks' frontiers (sra_classify_and_split_batch).
    nets / opts: one option set per network; frontier, out, leaves: CUDA int16
    [*, 4] node tensors; segs: BatchSeg list (or dicts of its fields).
    Returns counts, a CUDA int64 [len(segs), 8] tensor."""
    _need(frontier, torch.int16, 4, "frontier")
    segs = [s if isinstance(s, BatchSeg) else BatchSeg(**s) for s in segs]
    dev = frontier.device
    if counts is None:
        counts = torch.zeros((len(segs), CNT_N), dtype=torch.int64, device=dev)
    handles = (_vp * len(nets))(*[n.handle for n in nets])
    fo = (Opts * len(opts))(*opts)
    sg = (BatchSeg * len(segs))(*segs)
    _check(_lib.sra_classify_and_split_batch(handles, fo, len(nets), (C.c_float * 3)(*root_lo),
                                             (C.c_float * 3)(*root_hi), _ptr(frontier), sg, len(segs),
                                             _ptr(out), _ptr(leaves), _ptr(counts), _stream()))
    return counts


def mesh_leaves(net, leaves, sub_levels=3, root_lo=(-1.0, -1.0, -1.0), root_hi=(1.0, 1.0, 1.0), cap=None):
    """Marching-tetrahedra mesh of f = 0 inside the leaves (CUDA int16 [n,4]
    nodes), 2^sub_levels cells per leaf axis; returns CUDA float32 [T,3,3]."""
    _need(leaves, torch.int16, 4, "leaves")
    n = leaves.shape[0]
    cells = n * (1 << (3 * sub_levels))
    cap = cap if cap is not None else max(1, 2 * cells)
    tris = torch.empty((cap, 3, 3), dtype=torch.float32, device=leaves.device)
    nt = C.c_int64(0)
    code = _lib.sra_mesh_leaves(net.handle, (C.c_float * 3)(*root_lo), (C.c_float * 3)(*root_hi), _ptr(leaves), n,
                                int(sub_levels), _ptr(tris), int(cap), C.byref(nt), _stream())
    if code == ECAPACITY:
        return mesh_leaves(net, leaves, sub_levels, root_lo, root_hi, cap=int(nt.value))
    _check(code)
    return tris[:nt.value]


def empty_spheres(net, points, r_max=1.0, levels=12, opts=None, radius=None, **kw):
    """Empty-sphere radius per point (Sec. 4.4): the largest r_max * 2^-k whose
    box around the point is proven POSITIVE or NEGATIVE, else 0."""
    opts = opts or make_opts(**kw)
    _need(points, torch.float32, 3, "points")
    n = points.shape[0]
    radius = radius if radius is not None else torch.empty(n, dtype=torch.float32, device=points.device)
    _check(_lib.sra_empty_spheres(net.handle, C.byref(opts), _ptr(points), n, float(r_max), int(levels),
                                  _ptr(radius), _stream()))
    return radius


def cast_frustum(net, eye, dirs, width, height, grid=16, opts=None, **kw):
    """Frustum ray casting (Sec. 4.3) of a width x height pinhole image:
    dirs is a CUDA float32 [height*width, 3] tensor of unit pixel directions
    from eye. Returns (t_hit [H*W], iters [H*W], stats dict)."""
    opts = opts or make_opts(**kw)
    _need(dirs, torch.float32, 3, "dirs")
    n = width * height
    t_hit = torch.empty(n, dtype=torch.float32, device=dirs.device)
    iters = torch.empty(n, dtype=torch.int32, device=dirs.device)
    st = (C.c_int64 * 4)()
    _check(_lib.sra_cast_frustum(net.handle, C.byref(opts), (C.c_float * 3)(*[float(v) for v in eye]), _ptr(dirs),
                                 int(width), int(height), int(grid), _ptr(t_hit), _ptr(iters), st, _stream()))
    return t_hit, iters, {"rounds": st[0], "frustum_boxes": st[1], "rays": st[2]}


def cast_rays(net, origins, dirs, opts=None, t_hit=None, iters=None, **kw):
    """Proc. 2 per ray; returns (t_hit float32 [n], iters int32 [n]).

    precision "fp32" / "fp64" (SIMT) or "bf16" (tensor-core hidden layers);
    recheck=True marches again in FP64 every ray that met a segment bound
    within recheck_band of zero (recheck_count counts them)."""
    opts = opts or make_opts(**kw)
    _need(origins, torch.float32, 3, "origins")
    _need(dirs, torch.float32, 3, "dirs")
    n = origins.shape[0]
    dev = origins.device
    t_hit = t_hit if t_hit is not None else torch.empty(n, dtype=torch.float32, device=dev)
    iters = iters if iters is not None else torch.empty(n, dtype=torch.int32, device=dev)
    _check(_lib.sra_cast_rays(net.handle, C.byref(opts), _ptr(origins), _ptr(dirs), n,
                              _ptr(t_hit), _ptr(iters), _stream()))
    return t_hit, iters


def extract_leaves(net, depth, xl=(-1.0, -1.0, -1.0), xu=(1.0, 1.0, 1.0), opts=None, cap=None,
                   leaves=None, **kw):
    """Proc. 3 to a fixed depth; returns (leaves CUDA int16 [m,4], per-level counts [depth+1,3])."""
    opts = opts or make_opts(**kw)
    dev = torch.device("cuda", torch.cuda.current_device())
    if leaves is None:
        cap = cap if cap is not None else (1 << 20)
        leaves = torch.empty((max(cap, 1), 4), dtype=torch.int16, device=dev)
    cap = leaves.shape[0] if cap is None else cap
    nl = C.c_int64(0)
    lc = (C.c_int64 * (3 * (depth + 1)))()
    code = _lib.sra_extract_leaves(net.handle, C.byref(opts), (C.c_float * 3)(*xl),
                                   (C.c_float * 3)(*xu), int(depth), _ptr(leaves), int(cap),
                                   C.byref(nl), lc, _stream())
    if code == ECAPACITY:
        return extract_leaves(net, depth, xl, xu, opts, cap=int(nl.value))
    _check(code)
    counts = np.array(list(lc), np.int64).reshape(depth + 1, 3)
    return leaves[:nl.value], counts


def ray_request(net, form, arrival, origins, dirs, t_hit, iters=None):
    """A ray-tile query (Proc. 2) for serve(); the tensors must stay alive."""
    for t, nm in ((origins, "origins"), (dirs, "dirs")):
        _need(t, torch.float32, 3, nm)
    _need(t_hit, torch.float32, None, "t_hit")
    return Request(kind=REQ_RAYS, net=net, form=form, arrival=float(arrival), n=origins.shape[0],
                   a=_ptr(origins), b=_ptr(dirs), lo=_ptr(t_hit), iters=_ptr(iters))


def box_request(net, form, arrival, centers, halfw, lo, hi, cls=None):
    """A box-batch query (Proc. 1) for serve(); the tensors must stay alive."""
    _need(centers, torch.float32, 3, "centers")
    _need(halfw, torch.float32, 3, "halfw")
    return Request(kind=REQ_BOXES, net=net, form=form, arrival=float(arrival), n=centers.shape[0],
                   a=_ptr(centers), b=_ptr(halfw), lo=_ptr(lo), hi=_ptr(hi), cls=_ptr(cls))


def leaf_request(net, form, arrival, depth, leaves):
    """A leaf-extraction job (Proc. 3 to `depth`) for serve(); leaves is a
    CUDA int16 [cap, 4] tensor that also sets the capacity of each level's
    frontier buffer (the job reserves depth + 1 of them)."""
    return Request(kind=REQ_LEAVES, net=net, form=form, arrival=float(arrival), depth=int(depth),
                   leaves=_ptr(leaves), cap=leaves.shape[0])


def serve(nets, forms, requests, slots=4, frontier_bytes=256 << 20, realtime=True):
    """Run a request trace through sra_serve on the current device; the
    Request objects are filled in place (status, slot, t_admit, t_done,
    n_out, levels) and returned as a ctypes array."""
    torch.cuda.synchronize()
    arr = (Request * max(1, len(requests)))(*requests)
    handles = (_vp * len(nets))(*[n.handle for n in nets])
    fo = (Opts * len(forms))(*forms)
    cfg = ServeCfg(int(slots), int(bool(realtime)), int(frontier_bytes))
    _check(_lib.sra_serve(handles, len(nets), fo, len(forms), C.byref(cfg), arr, len(requests)))
    return arr[:len(requests)]
