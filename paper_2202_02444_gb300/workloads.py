"""Seeded synthetic inputs for the range-analysis path.

This module holds no range-analysis arithmetic. It only draws random networks,
boxes, octree nodes and camera rays, and it is the one module that both the
FP64 oracle tests and the CUDA path read their inputs from. The paper's own
workloads are trained shapes that are not available, so seeded random-init
networks stand in for them; the paper states its guarantees hold for
randomly initialised networks too (Sec. 1, Sec. 4.7).

Network parameter packing (shared by every consumer): for each linear layer
l = 0..L-1 the row-major weight W_l (widths[l+1] x widths[l]) followed by the
bias b_l (widths[l+1]), concatenated into one float32 vector.

Octree node records are four uint16 values (ix, iy, iz, level); see
``NODE_DTYPE``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ACT_IDENTITY, ACT_RELU, ACT_ELU, ACT_SIN = 0, 1, 2, 3
ACT_NAMES = {"identity": ACT_IDENTITY, "relu": ACT_RELU, "elu": ACT_ELU, "sin": ACT_SIN}

NODE_DTYPE = np.dtype([("ix", "<u2"), ("iy", "<u2"), ("iz", "<u2"), ("level", "<u2")])


@dataclass
class MLP:
    """A scalar MLP implicit function f: R^3 -> R.

    widths[0] is the network input width (3, or 3 + 6*octaves with the
    positional encoding), widths[-1] == 1. acts[l] is the activation after
    linear layer l for l < L-1; the last layer is linear.
    """

    widths: list
    acts: list
    params: np.ndarray  # float32, packed as described in the module docstring
    pe_octaves: int = 0
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_layers(self) -> int:
        return len(self.widths) - 1

    def layer(self, l):
        """(W, b) views of linear layer l."""
        off = 0
        for k in range(l):
            off += self.widths[k + 1] * self.widths[k] + self.widths[k + 1]
        o, i = self.widths[l + 1], self.widths[l]
        W = self.params[off:off + o * i].reshape(o, i)
        b = self.params[off + o * i:off + o * i + o]
        return W, b


def pe_width(octaves: int) -> int:
    """Input width after the sinusoidal encoding [x, sin(2^k pi x), cos(2^k pi x)]."""
    return 3 + 6 * octaves


def make_mlp(hidden, act="relu", seed=0, init=None, bias_std=0.1, pe_octaves=0,
             omega0=30.0, name=""):
    """Random-init MLP 3 -> hidden[0] -> ... -> hidden[-1] -> 1.

    init "he": W ~ N(0, 2/fan_in), b ~ N(0, bias_std^2) (bias_std is a standard
    deviation). init "siren": first layer U(+-1/fan_in), later layers
    U(+-sqrt(6/fan_in)/omega0); biases U(+-1/sqrt(fan_in)); the frequency omega0
    is folded into the weights and biases of every layer followed by sin, so the
    stored network is a plain sin-activated MLP. The last layer is linear.
    """
    if isinstance(act, str):
        act_code = ACT_NAMES[act]
    else:
        act_code = int(act)
    if init is None:
        init = "siren" if act_code == ACT_SIN else "he"
    rng = np.random.default_rng(seed)
    din = pe_width(pe_octaves) if pe_octaves else 3
    widths = [din] + list(hidden) + [1]
    L = len(widths) - 1
    acts = [act_code] * (L - 1)
    chunks = []
    for l in range(L):
        fi, fo = widths[l], widths[l + 1]
        if init == "he":
            W = rng.normal(0.0, math.sqrt(2.0 / fi), size=(fo, fi))
            b = rng.normal(0.0, bias_std, size=(fo,))
        elif init == "siren":
            lim = (1.0 / fi) if l == 0 else math.sqrt(6.0 / fi) / omega0
            W = rng.uniform(-lim, lim, size=(fo, fi))
            b = rng.uniform(-1.0 / math.sqrt(fi), 1.0 / math.sqrt(fi), size=(fo,))
            if l < L - 1 and acts[l] == ACT_SIN:
                W = W * omega0
                b = b * omega0
        else:
            raise ValueError(init)
        chunks.append(W.astype(np.float32).ravel())
        chunks.append(b.astype(np.float32).ravel())
    params = np.concatenate(chunks).astype(np.float32)
    return MLP(widths, acts, params, pe_octaves, name=name,
               meta={"seed": seed, "init": init, "act": act_code})


def make_custom_mlp(widths, acts, layers, pe_octaves=0, name=""):
    """MLP from explicit (W, b) float arrays (used for closed-form test nets)."""
    chunks = []
    for (W, b) in layers:
        chunks.append(np.asarray(W, np.float32).ravel())
        chunks.append(np.asarray(b, np.float32).ravel())
    return MLP(list(widths), list(acts), np.concatenate(chunks).astype(np.float32),
               pe_octaves, name=name)


# --- the named workloads -------------------------------------------------------

def net_small_relu():
    """ReLU 3-32-32-1, He-normal, bias std 0.1, seed 0."""
    return make_mlp([32, 32], "relu", seed=0, name="relu_3x32x32x1")


def net_relu256x8():
    """ReLU 3-[256]x8-1, He-normal, seed 1."""
    return make_mlp([256] * 8, "relu", seed=1, name="relu_3x256x8x1")


def net_elu512x6_pe():
    """ELU 39(PE, 6 octaves)-[512]x6-1, He-normal, seed 2."""
    return make_mlp([512] * 6, "elu", seed=2, pe_octaves=6, name="elu_pe6_512x6")


def net_batch_mix(i):
    """Network i (0..63) of the uneven multi-network batch (seeds 1000+i)."""
    rng = np.random.default_rng(1000 + i)
    width = int(rng.choice([32, 64, 128, 256, 512]))
    depth = int(rng.integers(3, 11))
    act = ["relu", "elu", "sin"][int(rng.integers(0, 3))]
    level = int(rng.integers(8, 12))
    net = make_mlp([width] * depth, act, seed=1000 + i, name=f"mix{i}_{act}_{width}x{depth}")
    net.meta["octree_depth"] = level
    return net


def make_boxes(n, seed=100, hw_lo=1.0 / 256, hw_hi=0.25):
    """n boxes: centers U[-1,1]^3, half-widths log-uniform in [hw_lo, hw_hi] per axis."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-1.0, 1.0, size=(n, 3)).astype(np.float32)
    halfw = np.exp(rng.uniform(math.log(hw_lo), math.log(hw_hi), size=(n, 3))).astype(np.float32)
    return centers, halfw


def random_nodes(n, level, seed=7):
    """n octree nodes drawn uniformly at one level (duplicates possible)."""
    rng = np.random.default_rng(seed)
    out = np.zeros(n, NODE_DTYPE)
    m = 1 << level
    out["ix"] = rng.integers(0, m, n)
    out["iy"] = rng.integers(0, m, n)
    out["iz"] = rng.integers(0, m, n)
    out["level"] = level
    return out


def root_node():
    out = np.zeros(1, NODE_DTYPE)
    return out


def camera_rays(width, height, eye=(0.0, 0.0, 3.0), target=(0.0, 0.0, 0.0),
                up=(0.0, 1.0, 0.0), vfov_deg=40.0):
    """Pinhole camera rays through pixel centres, row-major (y down), unit dirs."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    upv = np.cross(right, fwd)
    th = math.tan(math.radians(vfov_deg) * 0.5)
    aspect = width / height
    px = (np.arange(width) + 0.5) / width * 2.0 - 1.0
    py = 1.0 - (np.arange(height) + 0.5) / height * 2.0
    X, Y = np.meshgrid(px * th * aspect, py * th)
    d = fwd[None, None, :] + X[..., None] * right[None, None, :] + Y[..., None] * upv[None, None, :]
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    dirs = d.reshape(-1, 3).astype(np.float32)
    origins = np.broadcast_to(eye.astype(np.float32), dirs.shape).copy()
    return origins, dirs


def sphere_rays(n, seed=3, radius=3.0, jitter=0.5):
    """n rays from points on a sphere of the given radius, aimed near the origin."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    origins = (radius * v).astype(np.float32)
    tgt = rng.uniform(-jitter, jitter, size=(n, 3))
    d = tgt - origins
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return origins, d.astype(np.float32)


def sample_rows(n_total, n_sample, seed=11):
    """Sorted distinct indices of a seeded sample."""
    rng = np.random.default_rng(seed)
    n_sample = min(n_sample, n_total)
    return np.sort(rng.choice(n_total, size=n_sample, replace=False))
