"""Pins for the oracle's RangeBound (Proc. 1) and its arithmetic variants.

Checks, none of which trusts the oracle's own arithmetic:
  * the Sec. 3.1 worked example y = 2x - x (golden fixture, both readings);
  * exactness of affine arithmetic on affine networks (corner brute force:
    the extremes of an affine map over a box sit at its corners, Sec. 3.2);
  * soundness against dense point samples evaluated by an independent numpy
    forward pass (the fuzz test of Sec. 3.6), for every policy and activation,
    with and without positional encoding;
  * affine-truncate with K >= all symbols equals affine-full (Sec. 3.3);
  * the oracle's plain evaluator equals the numpy forward pass.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2202_02444_gb300 import workloads as wl
from tests.np_forward import box_samples, forward

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_dependency_example_golden():
    d = json.load(open(os.path.join(GOLDEN, "dependency_2x_minus_x.json")))
    n = d["net"]
    net = wl.make_custom_mlp(n["widths"], [0], [(n["W1"], n["b1"]), (n["W2"], n["b2"])])
    for case in d["cases"]:
        a, b = case["x"]
        c = np.array([(a + b) / 2, 0.0, 0.0])
        ax = np.array([[(b - a) / 2, 0.0, 0.0]])
        _, lo, hi, _, _ = oracle.range_bound(net, c, ax, "interval")
        assert (lo, hi) == tuple(case["interval"])
        for arith in ("fixed", "full", "truncate"):
            _, lo, hi, _, _ = oracle.range_bound(net, c, ax, arith, K=4)
            assert (lo, hi) == pytest.approx(tuple(case["affine"]), abs=1e-15)


def affine_net(seed, depth=3, width=8):
    """Random net with identity activations: an affine map."""
    rng = np.random.default_rng(seed)
    widths = [3] + [width] * depth + [1]
    layers = [(rng.normal(size=(widths[i + 1], widths[i])), rng.normal(size=widths[i + 1]))
              for i in range(len(widths) - 1)]
    return wl.make_custom_mlp(widths, [0] * depth, layers)


@pytest.mark.parametrize("seed", range(5))
def test_affine_exact_on_affine_networks(seed):
    net = affine_net(seed)
    c, h = wl.make_boxes(64, seed=seed)
    corners = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)], float)
    for arith in ("fixed", "truncate", "full"):
        r = oracle.bound_boxes(net, c, h, arith, K=3)
        for i in range(len(c)):
            ys = forward(net, c[i] + corners * h[i])
            scale = 1 + np.abs(ys).max()
            assert r["lo"][i] == pytest.approx(ys.min(), abs=1e-12 * scale)
            assert r["hi"][i] == pytest.approx(ys.max(), abs=1e-12 * scale)


def test_single_linear_layer_exact():
    """One linear layer: range = w.c + b +- sum_i |w_i| h_i (Sec. 3.2)."""
    rng = np.random.default_rng(5)
    w, b = rng.normal(size=(1, 3)), rng.normal(size=1)
    net = wl.make_custom_mlp([3, 1], [], [(w, b)])
    c, h = wl.make_boxes(32, seed=9)
    r = oracle.bound_boxes(net, c, h, "fixed")
    w32 = w.astype(np.float32).astype(np.float64)[0]
    b32 = float(np.float32(b[0]))
    for i in range(32):
        mid = float(w32 @ c[i].astype(np.float64)) + b32
        rad = float(np.abs(w32) @ h[i].astype(np.float64))
        assert r["lo"][i] == pytest.approx(mid - rad, abs=1e-13)
        assert r["hi"][i] == pytest.approx(mid + rad, abs=1e-13)
        # interval arithmetic is also exact on a single linear layer
    ri = oracle.bound_boxes(net, c, h, "interval")
    np.testing.assert_allclose(ri["lo"], r["lo"], atol=1e-13)
    np.testing.assert_allclose(ri["hi"], r["hi"], atol=1e-13)


NETS = {
    "relu": lambda: wl.make_mlp([16, 16, 16], "relu", seed=21),
    "elu": lambda: wl.make_mlp([16, 16, 16], "elu", seed=22),
    "sin": lambda: wl.make_mlp([16, 16], "sin", seed=23),
    "elu_pe": lambda: wl.make_mlp([16, 16], "elu", seed=24, pe_octaves=2),
    "small": wl.net_small_relu,
}


@pytest.mark.parametrize("name", list(NETS))
@pytest.mark.parametrize("arith,K", [("interval", 0), ("fixed", 0), ("truncate", 4),
                                     ("truncate", 12), ("full", 0)])
@pytest.mark.parametrize("slope", ["chebyshev", "minrange"])
def test_soundness_brute_force(name, arith, K, slope):
    """Every sampled f(x) lies inside [lo, hi] (the fuzz test of Sec. 3.6)."""
    net = NETS[name]()
    hw_hi = 0.25 if name not in ("sin", "elu_pe") else 0.05
    c, h = wl.make_boxes(48, seed=hash((name, arith, K)) % 1000, hw_hi=hw_hi)
    r = oracle.bound_boxes(net, c, h, arith, K=K, slope=slope)
    for i in range(len(c)):
        ys = forward(net, box_samples(c[i], h[i], seed=i))
        tol = 1e-10 * (1 + np.abs(ys).max())
        assert ys.min() >= r["lo"][i] - tol, (i, ys.min(), r["lo"][i])
        assert ys.max() <= r["hi"][i] + tol, (i, ys.max(), r["hi"][i])
        assert r["rad"][i] >= 0


def test_truncate_with_room_for_all_symbols_equals_full():
    net = NETS["small"]()
    c, h = wl.make_boxes(64, seed=4)
    full = oracle.bound_boxes(net, c, h, "full")
    trunc = oracle.bound_boxes(net, c, h, "truncate", K=3 + 32 + 32)
    np.testing.assert_array_equal(full["lo"], trunc["lo"])
    np.testing.assert_array_equal(full["hi"], trunc["hi"])


def cancel_net():
    """Hand-built ReLU net: h1 = ReLU(0.1 x0), h2 = ReLU(x0); g1 = g2 = h2 + 10
    (always active); y = g1 - g2 == 0. On x0 in [-1,1] the first layer makes
    new symbols of size 0.025 (row h1, candidate 1) and 0.25 (row h2,
    candidate 2) next to the input symbol column [0.05, 0.5] (candidate 0).
    The large new symbol is not the first one, so keeping columns by index
    and keeping them by size differ."""
    W1 = np.array([[0.1, 0, 0], [1.0, 0, 0]]); b1 = np.zeros(2)
    W2 = np.array([[0.0, 1.0], [0.0, 1.0]]); b2 = np.array([10.0, 10.0])
    W3 = np.array([[1.0, -1.0]]); b3 = np.zeros(1)
    return wl.make_custom_mlp([3, 2, 2, 1], [1, 1], [(W1, b1), (W2, b2), (W3, b3)])


@pytest.mark.parametrize("arith,K,expect", [
    ("interval", 0, (-1.0, 1.0)),
    ("fixed", 0, (-0.5, 0.5)),
    ("truncate", 1, (-0.5, 0.5)),   # keeps only the input column
    ("truncate", 2, (0.0, 0.0)),    # keeps the input column and the 0.25 symbol
    ("truncate", 3, (0.0, 0.0)),
    ("full", 0, (0.0, 0.0)),
])
def test_condense_policies_closed_form(arith, K, expect):
    """Sec. 3.3 policies on a net whose exact output is 0. Keeping the large
    new symbol lets it cancel through the two paths; condensing it into the
    per-component x_inf (App. A) cannot cancel (0.25 + 0.25 = 0.5). A
    truncate that kept the first or the smallest columns fails at K=2."""
    net = cancel_net()
    _, lo, hi, _, _ = oracle.range_bound(net, [0.0, 0, 0], [[1.0, 0, 0]], arith, K=K)
    assert (lo, hi) == pytest.approx(expect, abs=1e-6)


def test_more_symbols_tighter_on_average():
    """Table 1 ordering of the decided lengths: full >= truncate >= fixed in
    tightness (compared as mean widths; not a per-box law)."""
    net = NETS["relu"]()
    c, h = wl.make_boxes(64, seed=8)
    full = oracle.bound_boxes(net, c, h, "full")
    t12 = oracle.bound_boxes(net, c, h, "truncate", K=12)
    fixed = oracle.bound_boxes(net, c, h, "fixed")
    w_full = (full["hi"] - full["lo"]).mean()
    w_t = (t12["hi"] - t12["lo"]).mean()
    w_fix = (fixed["hi"] - fixed["lo"]).mean()
    assert w_full <= w_t * 1.0001 and w_t <= w_fix * 1.0001


def test_affine_tighter_than_interval_in_aggregate():
    """Sec. 3.1/3.2, Table 1: interval bounds are far looser on multi-layer
    nets. Per box this need not hold (ReLU on [-1,1]), so compare means."""
    net = wl.net_small_relu()
    c, h = wl.make_boxes(256, seed=100)
    a = oracle.bound_boxes(net, c, h, "fixed")
    i = oracle.bound_boxes(net, c, h, "interval")
    assert (a["hi"] - a["lo"]).mean() < 0.7 * (i["hi"] - i["lo"]).mean()


def test_classification_strict():
    """Proc. 1: POSITIVE iff lo > 0, NEGATIVE iff hi < 0 (a bound touching 0
    is UNKNOWN). Net f(x) = x0 on boxes [0, 2] and [-2, 0]."""
    net = wl.make_custom_mlp([3, 1], [], [(np.array([[1.0, 0, 0]]), np.array([0.0]))])
    cls, lo, hi, _, _ = oracle.range_bound(net, [1.0, 0, 0], [[1.0, 0, 0]])
    assert lo == 0.0 and cls == oracle.UNKNOWN
    cls, lo, hi, _, _ = oracle.range_bound(net, [-1.0, 0, 0], [[1.0, 0, 0]])
    assert hi == 0.0 and cls == oracle.UNKNOWN
    cls, *_ = oracle.range_bound(net, [1.5, 0, 0], [[1.0, 0, 0]])
    assert cls == oracle.POSITIVE


@pytest.mark.parametrize("name", ["relu", "elu_pe", "sin"])
def test_plain_eval_matches_numpy(name):
    net = NETS[name]()
    x = np.random.default_rng(0).uniform(-1, 1, size=(200, 3))
    np.testing.assert_allclose(oracle.evaluate(net, x), forward(net, x), rtol=1e-12, atol=1e-12)
