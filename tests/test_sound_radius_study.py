"""Where a sound bound has to keep its rounding errors: a pinned FP64 study on
the ReLU 3-[256]x8-1 network (He init, seed 1) with affine-truncate K = 64,
over 64 uniformly drawn level-7 octree nodes.

The paper computes without rounding control (Sec. 3.4). A bound that is
guaranteed in floating point has to add, after every dense layer, a radius
rho that covers that layer's rounding errors. The tensor-core kernel of this
library (precision BF16_SOUND) bounds them a priori by u = 8.07e-5 per unit
of |W| (|c| + |A|) for H = 256 (BF16 hi/lo products: 2^-16; FP32
accumulation over 32 sixteen-deep MMA steps: 17 * 2^-23 each) and puts rho in
x_inf, which every later layer multiplies by |W| (it also adds the BF16
rounding of the stored noise entries, 2^-8 of their magnitudes; with both
terms the emulation reproduces the kernel's UNKNOWN fractions on shallower
networks, tests/test_gpu_bf16.py). On this network the first term alone
leaves every box UNKNOWN. The emulation (tests/sound_emulation.py, pinned here to the
C oracle) measures the UNKNOWN fraction of each way of carrying rho, for
per-layer relative errors u (the exact bound leaves 2 of the 64 nodes, 0.031,
UNKNOWN):

  scheme                                       u=8.07e-5  6e-6   1e-7   1e-9
  rho in x_inf (the kernel's scheme)              1.00    1.00   1.00   0.031
  rho as new symbols competing in the top-64      1.00    1.00   0.98   0.031
  rho as symbols kept for 2 layers, then x_inf    1.00    1.00   0.031  0.031
  rho as symbols kept for 5 layers                0.094   0.031    -      -
  rho as symbols never dropped (full errors)      0.047   0.031    -      -

So a sound bound that decides what the oracle decides on this network needs
either rounding errors near 1e-9 (FP64-like arithmetic), or FP32-like errors
(1e-7) with every layer's errors carried as their own noise symbols for two
layers, or the kernel's errors carried for five: 256 to 1280 extra columns
per box, against the 64 columns of the bound itself. The BF16-sound kernel
does neither: it stays sound, and its classes are gated against the oracle on
shallower networks (tests/test_gpu_bf16.py).
"""
import numpy as np
import pytest

import oracle
from paper_2202_02444_gb300 import workloads as wl
from tests.sound_emulation import bound, node_boxes

U_KERNEL = (2.0 ** -16 + 17 * 32 * 2.0 ** -23 * (1 + 2.0 ** -7)) * 1.001  # 8.07e-5


@pytest.fixture(scope="module")
def case():
    mlp = wl.net_relu256x8()
    nodes = wl.random_nodes(64, level=7, seed=21)
    c, h = node_boxes(nodes)
    cls0, lo0, hi0, rad0 = bound(mlp, c, h, 64)
    return mlp, nodes, c, h, cls0, lo0, hi0, rad0


def unknown(cls):
    return float(np.mean(cls == 0))


def test_emulation_is_the_oracle_without_rounding(case):
    """u = 0: the emulation is affine-truncate itself (same classes and bounds
    as the C oracle, which is pinned by its own tests)."""
    mlp, nodes, c, h, cls0, lo0, hi0, rad0 = case
    ocls, olo, ohi, _ = oracle.classify_nodes(mlp, nodes, (-1, -1, -1), (1, 1, 1), oracle.OCTREE,
                                              "truncate", K=64)
    assert np.array_equal(ocls, cls0)
    scale = np.abs(0.5 * (olo + ohi)) + 0.5 * (ohi - olo)
    assert np.all(np.abs(olo - lo0) <= 1e-9 * scale) and np.all(np.abs(ohi - hi0) <= 1e-9 * scale)
    assert 0.0 < unknown(cls0) < 0.1


def test_radius_in_x_inf_decides_nothing(case):
    mlp, nodes, c, h, cls0, *_ = case
    for u in (U_KERNEL, 6e-6, 1e-7):
        assert unknown(bound(mlp, c, h, 64, "xinf", u)[0]) == 1.0
    cls9 = bound(mlp, c, h, 64, "xinf", 1e-9)[0]
    assert np.array_equal(cls9, cls0)  # FP64-like errors: the oracle's classes


def test_radius_as_competing_symbols_does_not_help(case):
    mlp, nodes, c, h, cls0, *_ = case
    assert unknown(bound(mlp, c, h, 64, "sym", U_KERNEL)[0]) == 1.0
    assert unknown(bound(mlp, c, h, 64, "sym", 1e-7)[0]) >= 0.9


def test_radius_as_kept_symbols(case):
    mlp, nodes, c, h, cls0, lo0, hi0, rad0 = case
    assert unknown(bound(mlp, c, h, 64, "delay", U_KERNEL, d=2)[0]) == 1.0
    assert np.array_equal(bound(mlp, c, h, 64, "delay", 1e-7, d=2)[0], cls0)
    assert unknown(bound(mlp, c, h, 64, "delay", U_KERNEL, d=5)[0]) <= unknown(cls0) + 4 / 64
    assert np.array_equal(bound(mlp, c, h, 64, "delay", 6e-6, d=5)[0], cls0)
    cls_k, lo_k, hi_k, rad_k = bound(mlp, c, h, 64, "delay", U_KERNEL, d=None)
    assert unknown(cls_k) <= unknown(cls0) + 1 / 64
    # the radius only widens the exact-arithmetic bound
    assert np.all(rad_k >= rad0 * (1 - 1e-12))


@pytest.mark.parametrize("act,seed", [("elu", 36), ("sin", 38)])
def test_emulation_elu_sin_is_the_oracle_without_rounding(act, seed):
    """The emulation's ELU and sin rules and truncation on an ELU and a
    SIREN network equal the oracle's (the model the BF16-sound ELU and sin
    gates of tests/test_gpu_bf16.py use)."""
    mlp = wl.make_mlp([128] * 3, act, seed=seed)
    c, h = wl.make_boxes(96, seed=7, hw_lo=1 / 256, hw_hi=1 / 16)
    cls0, lo0, hi0, rad0 = bound(mlp, c.astype(np.float64), h.astype(np.float64), 64)
    ref = oracle.bound_boxes(mlp, c, h, "truncate", K=64)
    scale = np.abs(ref["y0"]) + ref["rad"]
    tie = ref["sel_gap"] < 1e-6
    assert np.all(((np.abs(ref["lo"] - lo0) <= 1e-9 * scale) & (np.abs(ref["hi"] - hi0) <= 1e-9 * scale)) | tie)
    assert np.all((cls0 == ref["cls"]) | tie)


def test_emulation_sin_rule_is_the_oracle_rule():
    """The emulation's vectorised sin rule against the oracle's, range by
    range: ranges of every length up to 3 pi (at and past 2 pi the slope is
    0), ranges with an end on a critical point or a multiple of pi, and
    ranges far from the origin."""
    from tests.sound_emulation import _sin_rule
    rng = np.random.default_rng(5)
    c = np.concatenate([rng.uniform(-40, 40, 400), np.pi * np.arange(-6, 7), np.full(6, 0.5 * np.pi)])
    r = np.concatenate([rng.uniform(0, 1.5 * np.pi, 400), np.full(13, 0.3), [0.0, 1e-9, np.pi / 2, np.pi, 1.2 * np.pi,
                                                                               3.0]])
    a, b, g = _sin_rule(c, r)
    for i in range(len(c)):
        ra, rb, rg = oracle.linearize(wl.ACT_SIN, c[i] - r[i], c[i] + r[i])
        assert abs(a[i] - ra) <= 1e-12 and abs(b[i] - rb) <= 1e-9 * (1 + abs(c[i])) and abs(g[i] - rg) <= 1e-9
