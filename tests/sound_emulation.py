"""FP64 emulation of affine-truncate RangeBound with an injected rounding
radius: a study of where a sound (rounding-aware) bound has to keep its
rounding errors.

TEST INFRASTRUCTURE (numpy, FP64). It follows the same steps as the oracle
(Proc. 1; App. A Table "affine_update_rules"; the ReLU, ELU and sin rules of
Table "affine_nonlinearities" with the Chebyshev slope; Sec. 3.3 truncate: K old
plus the new columns scored by their L1 norm, ties to the lower index,
dropped magnitudes added to x_inf row by row) and adds, after every dense
layer but the first, a per-neuron radius

    rho_i = u * sum_j |W_ij| (|c_j| + sum_k |A_jk|)

that bounds the rounding error of the layer's FP operations when every
product and sum has relative error u (c the centre, A the noise columns).
Where that radius goes is the scheme:

  * "xinf":  into x_inf (the independent per-component term of App. A);
  * "sym":   as one new noise symbol per neuron that competes in the top-K of
             Sec. 3.3 with the activation symbols;
  * "delay": as one new noise symbol per neuron kept outside the top-K for
             `d` layers, then condensed into x_inf (d = None: never).

With u = 0 every scheme is the plain affine-truncate bound of the oracle.
"""
from __future__ import annotations

import numpy as np


def node_boxes(nodes):
    """Centres and half-widths of octree nodes of [-1, 1]^3."""
    w = 2.0 / (1 << nodes["level"].astype(np.int64))
    lo = -1.0 + np.stack([nodes["ix"], nodes["iy"], nodes["iz"]], 1) * w[:, None]
    return lo + 0.5 * w[:, None], np.repeat((0.5 * w)[:, None], 3, 1)


def _relu_rule(c, r):
    lo, hi = c - r, c + r
    mixed = (lo < 0) & (hi > 0)
    den = np.where(mixed, hi - lo, 1.0)
    al = np.where(hi <= 0, 0.0, np.where(lo >= 0, 1.0, hi / den))
    be = np.where(mixed, -al * lo / 2, 0.0)
    return al, be, be


def _elu(x):
    return np.where(x > 0, x, np.expm1(np.minimum(x, 0.0)))


def _elu_rule(c, r):
    """ELU's rule (App. A, reading R2): the secant slope, the secant and
    tangent intercepts; the identity where the range is non-negative."""
    lo, hi = c - r, c + r
    w = hi - lo
    a = np.where(w > 0, (_elu(hi) - _elu(lo)) / np.where(w > 0, w, 1.0), np.exp(np.minimum(lo, 0.0)))
    ru = _elu(lo) - a * lo
    rl = np.where(a > 0, (a - 1) - a * np.log(np.where(a > 0, a, 1.0)), -1.0)
    b = (ru + rl) / 2
    ident = lo >= 0
    return np.where(ident, 1.0, a), np.where(ident, 0.0, b), np.where(ident, 0.0, ru - b)


def _cos_range(lo, hi):
    """Range of cos on [lo, hi] (App. A): the ends, and +-1 wherever a
    maximum 2 pi k or a minimum pi + 2 pi k lies inside."""
    tp = 2 * np.pi
    cl, cu = np.cos(lo), np.cos(hi)
    top = np.where(tp * np.ceil(lo / tp) <= hi, 1.0, np.maximum(cl, cu))
    bot = np.where(tp * np.ceil((lo - np.pi) / tp) + np.pi <= hi, -1.0, np.minimum(cl, cu))
    full = hi - lo >= tp
    return np.where(full, -1.0, bot), np.where(full, 1.0, top)


def _sin_rule(c, r):
    """sin's rule (App. A, reading R3): the slope is the mid-point of the cos
    range; g(x) = sin(x) - alpha x is bounded over the ends and the extreme
    critical points +-acos(alpha) + 2 pi k of both families in [lo, hi]."""
    lo, hi = c - r, c + r
    tp = 2 * np.pi
    sl, su = _cos_range(lo, hi)
    a = (sl + su) / 2
    ep = np.arccos(np.clip(a, -1.0, 1.0))
    cand = [lo, hi]
    for f in (ep, -ep):
        cand.append(np.clip(f + tp * np.ceil((lo - f) / tp), lo, hi))
        cand.append(np.clip(f + tp * np.floor((hi - f) / tp), lo, hi))
    g = np.stack([np.sin(x) - a * x for x in cand])
    ru, rl = g.max(0), g.min(0)
    b = (ru + rl) / 2
    return a, b, ru - b


RULES = {1: _relu_rule, 2: _elu_rule, 3: _sin_rule}


def _truncate(A, new, K):
    C = np.concatenate([A, new], axis=2)
    B, h, m = C.shape
    if m <= K:
        return np.concatenate([C, np.zeros((B, h, K - m))], 2), np.zeros((B, h))
    score = np.abs(C).sum(axis=1)
    keep = np.sort(np.argsort(-score, axis=1, kind="stable")[:, :K], axis=1)
    mask = np.zeros((B, m), bool)
    np.put_along_axis(mask, keep, True, axis=1)
    kept = np.take_along_axis(C, keep[:, None, :], axis=2)
    return kept, (np.abs(C) * (~mask)[:, None, :]).sum(axis=2)


def bound(mlp, centers, halfw, K, scheme="xinf", u=0.0, d=None, u_store=0.0, u_first=0.0):
    """Affine-truncate bound of a ReLU, ELU or sin MLP (its first activation
    decides) over boxes, with the rounding radius of `scheme`. u_store > 0 adds, after each hidden activation,
    u_store * alpha_i * sum_k |A_ik| to x_inf: the rounding of the scaled noise
    entries when they are stored in a narrower format for the next layer
    (BF16: u_store = 2^-8). u_first > 0 adds to x_inf of the first layer
    u_first * (|b| + |W| |c|) + (u_first / 2) * |W| |A|: the error of a
    three-term FP32 dot product and of the rounded products (u_first =
    2^-22). Returns (cls, lo, hi, rad): cls 1 POSITIVE,
    2 NEGATIVE, 0 UNKNOWN."""
    L, B = mlp.n_layers, len(centers)
    rule = RULES[int(mlp.acts[0])]
    c = np.asarray(centers, np.float64)
    A = np.zeros((B, 3, 3))
    A[:, [0, 1, 2], [0, 1, 2]] = np.asarray(halfw, np.float64)
    xi = np.zeros((B, 3))
    errs = []  # delay scheme: [age, columns]
    for l in range(L):
        W, b = (x.astype(np.float64) for x in mlp.layer(l))
        aW = np.abs(W)
        esum = sum(np.abs(E).sum(2) for _, E in errs) if errs else 0.0
        rho = u * ((np.abs(c) + np.abs(A).sum(2) + esum) @ aW.T) if (l > 0 and u > 0) else None
        c0 = c
        c = c @ W.T + b
        A = np.einsum("oi,bik->bok", W, A)
        errs = [[a, np.einsum("oi,bik->bok", W, E)] for a, E in errs]
        xi = xi @ aW.T
        if l == 0 and u_first > 0:
            xi = xi + u_first * (np.abs(b) + np.abs(c0) @ aW.T) + 0.5 * u_first * np.abs(A).sum(2)
        if l == L - 1:
            if rho is not None:
                xi = xi + rho
            break
        esum = sum(np.abs(E).sum(2) for _, E in errs) if errs else 0.0
        r = np.abs(A).sum(2) + xi + esum + (rho if rho is not None else 0.0)
        al, be, ga = rule(c, r)
        if u_store > 0:
            xi = xi + u_store * np.abs(A).sum(2)  # becomes |al| * (...) below
        c = al * c + be
        A = al[:, :, None] * A
        xi = np.abs(al) * xi  # sin's slope may be negative
        errs = [[a + 1, al[:, :, None] * E] for a, E in errs]
        h = c.shape[1]
        idx = np.arange(h)
        new = np.zeros((B, h, h))
        new[:, idx, idx] = ga
        if rho is not None:
            er = np.zeros((B, h, h))
            er[:, idx, idx] = np.abs(al) * rho
            if scheme == "xinf":
                xi = xi + np.abs(al) * rho
            elif scheme == "sym":
                new = np.concatenate([new, er], 2)
            elif scheme == "delay":
                errs.append([0, er])
            else:
                raise ValueError(scheme)
        if d is not None:
            kept = []
            for a, E in errs:
                if a >= d:
                    xi = xi + np.abs(E).sum(2)
                else:
                    kept.append([a, E])
            errs = kept
        A, drop = _truncate(A, new, K)
        xi = xi + drop
    y0 = c[:, 0]
    rad = np.abs(A[:, 0, :]).sum(1) + xi[:, 0] + sum(np.abs(E[:, 0, :]).sum(1) for _, E in errs)
    lo, hi = y0 - rad, y0 + rad
    return np.where(lo > 0, 1, np.where(hi < 0, 2, 0)), lo, hi, rad
