"""How far plain FP32 arithmetic drifts from the FP64 oracle on the
39(PE, 6 octaves)-[512]x6-1 ELU network (affine-fixed), on segment-sized
boxes and on boxes whose bound grows to radii of 1e3..1e7 through the six
512-wide layers: the basis of the 1e-5 FP32 gate of the GPU parity test of
that network (tests/test_gpu_boxes.py, test_elu512x6_pe_fixed_sample).

A float32 emulation of the same bound runs here on the CPU: the encoding rows
and every activation rule (Sec. 3.2, App. A tables "affine_update_rules" and
"affine_nonlinearities") in FP64 through the oracle's rule and rounded to
float32, and every dense layer as float32 dot products summed in input order
with one rounding per fused multiply-add (a thread of the SIMT engine sums its
row that way). Affine-fixed keeps the three box symbols and moves every new
symbol to x_inf. On both box sizes these float32 sums stay within 1e-5 of
|center| + radius of the FP64 bound (measured: below 1e-6), so the FP32 form
has no reason to be held to a looser gate.
"""
import numpy as np
import pytest

import oracle
from paper_2202_02444_gb300 import workloads as wl

SIN, ELU = 3, 2


def fma_rows(W, x):
    """y[b, o] = sum_j W[o, j] x[b, j, ...] in float32, in input order, one
    rounding per step (the product of two floats is exact in float64)."""
    W64 = W.astype(np.float64)
    acc = np.zeros((x.shape[0], W.shape[0]) + x.shape[2:], np.float32)
    for j in range(W.shape[1]):
        w = W64[:, j].reshape((1, -1) + (1,) * (x.ndim - 2))
        acc = (acc.astype(np.float64) + w * x[:, j:j + 1].astype(np.float64)).astype(np.float32)
    return acc


def rule(act, lo, hi):
    al, be, ga = (np.empty(lo.shape) for _ in range(3))
    for idx in np.ndindex(lo.shape):
        al[idx], be[idx], ga[idx] = oracle.linearize(act, float(lo[idx]), float(hi[idx]))
    return al, be, ga


def fixed_bound_fp32(mlp, c, h):
    B, oc = len(c), mlp.pe_octaves
    m = 3 + 6 * oc
    C, A, X = np.zeros((B, m)), np.zeros((B, m, 3)), np.zeros((B, m))
    for i in range(m):  # the encoding (R8), FP64
        if i < 3:
            C[:, i], A[:, i, i] = c[:, i], h[:, i]
            continue
        q = i - 3
        k, d, shift = q // 6, q % 3, (np.pi / 2 if q % 6 >= 3 else 0.0)
        s = np.ldexp(np.pi, k)
        pc, pa = s * c[:, d].astype(np.float64) + shift, s * h[:, d].astype(np.float64)
        al, be, ga = rule(SIN, pc - np.abs(pa), pc + np.abs(pa))
        C[:, i], A[:, i, d], X[:, i] = al * pc + be, al * pa, np.abs(ga)
    C, A, X = C.astype(np.float32), A.astype(np.float32), X.astype(np.float32)
    for l in range(mlp.n_layers):
        W, b = mlp.layer(l)
        C = (fma_rows(W, C).astype(np.float64) + b).astype(np.float32)
        A = fma_rows(W, A)
        X = fma_rows(np.abs(W), X)
        if l == mlp.n_layers - 1:
            break
        r = (np.abs(A).astype(np.float64).sum(2) + X).astype(np.float32)
        al, be, ga = rule(ELU, (C - r).astype(np.float64), (C + r).astype(np.float64))
        al, be, ga = al.astype(np.float32), be.astype(np.float32), ga.astype(np.float32)
        C = (al * C + be).astype(np.float32)
        A = (al[:, :, None] * A).astype(np.float32)
        X = (np.abs(al) * X + np.abs(ga)).astype(np.float32)
    return C[:, 0].astype(np.float64), np.abs(A[:, 0]).astype(np.float64).sum(1) + X[:, 0]


@pytest.fixture(scope="module")
def mlp():
    return wl.net_elu512x6_pe()


@pytest.mark.parametrize("hw_lo,hw_hi", [(1e-5, 1e-3), (1e-3, 1e-2)])
def test_fp32_drift_against_fp64(mlp, hw_lo, hw_hi):
    c, h = wl.make_boxes(24, seed=12, hw_lo=hw_lo, hw_hi=hw_hi)
    ref = oracle.bound_boxes(mlp, c, h, "fixed")
    y0, rad = fixed_bound_fp32(mlp, c, h)
    scale = np.abs(ref["y0"]) + ref["rad"]
    drift = np.maximum(np.abs(y0 - ref["y0"]), np.abs(rad - ref["rad"])) / scale
    print(f"half-widths [{hw_lo}, {hw_hi}]: FP32 drift / scale median {np.median(drift):.2e} max {drift.max():.2e}")
    assert drift.max() < 1e-5
