"""Pins for the oracle's scalar rules (App. A Table "affine_nonlinearities",
Sec. 3.1 interval rules) against brute force, closed forms and optimality.

No expected value here comes from the oracle itself: every check compares the
oracle's alpha/beta/gamma against a dense evaluation of the activation written
out in numpy, or against a closed form stated in the test.
"""
import math

import numpy as np
import pytest

import oracle

RELU, ELU, SIN = 1, 2, 3


def f_np(act, x):
    if act == RELU:
        return np.maximum(x, 0.0)
    if act == ELU:
        return np.where(x > 0, x, np.expm1(np.minimum(x, 0.0)))
    if act == SIN:
        return np.sin(x)
    raise ValueError(act)


def dense(l, u, n=20001):
    xs = np.linspace(l, u, n)
    # add the points where derivatives change or extrema sit
    extra = [0.0]
    if u - l < 200:
        k0, k1 = math.floor(l / (math.pi / 2)) - 1, math.ceil(u / (math.pi / 2)) + 1
        extra += [k * math.pi / 2 for k in range(k0, k1 + 1)]
    ex = np.array([e for e in extra if l <= e <= u])
    return np.concatenate([xs, ex])


def max_err(act, a, b, l, u):
    xs = dense(l, u)
    g = f_np(act, xs) - (a * xs + b)
    return g.max(), g.min()


def intervals(seed, n, scale):
    rng = np.random.default_rng(seed)
    c = rng.normal(0, scale, n)
    r = np.exp(rng.uniform(math.log(1e-4), math.log(3 * scale), n))
    return list(zip(c - r, c + r))


@pytest.mark.parametrize("act", [RELU, ELU, SIN])
@pytest.mark.parametrize("slope", ["chebyshev", "minrange"])
def test_linearisation_is_sound_and_tight(act, slope):
    """|f(x) - alpha x - beta| <= gamma on [l,u] (Eq. affine_func_update), and
    gamma is attained: the rule's beta, gamma are the exact extremes of
    f(x) - alpha x (both the ReLU/ELU Chebyshev form and the sin form)."""
    for (l, u) in intervals(1 + act, 400, 2.0 if act != SIN else 6.0):
        a, b, g = oracle.linearize(act, l, u, slope)
        hi, lo = max_err(act, a, b, l, u)
        tol = 1e-9 * (1 + abs(a) * max(abs(l), abs(u)))
        assert hi <= g + tol and lo >= -g - tol, (act, l, u, a, b, g, hi, lo)
        assert g >= 0
        # attained: dense grid spacing limits how close we get
        assert hi >= g - 1e-6 * (u - l) - tol and lo <= -g + 1e-6 * (u - l) + tol, (l, u, g, hi, lo)


@pytest.mark.parametrize("act", [RELU, ELU])
def test_chebyshev_is_minimax(act):
    """For convex ReLU/ELU the Chebyshev line minimises the max error: any
    other slope, with its best offset, has error >= gamma."""
    for (l, u) in intervals(11 + act, 100, 2.0):
        if u <= 0 and act == RELU or l >= 0:
            continue
        a, b, g = oracle.linearize(act, l, u)
        for da in (-0.05, -0.01, 0.01, 0.05):
            hi, lo = max_err(act, a + da, 0.0, l, u)
            assert (hi - lo) / 2 >= g - 1e-9


def test_relu_closed_form_and_special_cases():
    """Table ReLU row: alpha = u/(u-l), beta = gamma = -alpha l / 2; zero map
    for u <= 0; identity for l >= 0."""
    for (l, u) in [(-1.0, 1.0), (-3.0, 0.5), (-0.25, 4.0)]:
        a, b, g = oracle.linearize(RELU, l, u)
        assert a == pytest.approx(u / (u - l), rel=1e-15)
        assert b == pytest.approx(-a * l / 2, rel=1e-15)
        assert g == pytest.approx(-a * l / 2, rel=1e-15)
    assert oracle.linearize(RELU, -2.0, -1.0) == (0.0, 0.0, 0.0)
    assert oracle.linearize(RELU, -2.0, 0.0) == (0.0, 0.0, 0.0)
    assert oracle.linearize(RELU, 0.0, 3.0) == (1.0, 0.0, 0.0)
    assert oracle.linearize(RELU, 1.0, 1.0) == (1.0, 0.0, 0.0)
    # ReLU on [-1,1]: the counterexample to "interval contains affine"
    assert oracle.linearize(RELU, -1.0, 1.0) == (0.5, 0.25, 0.25)


def test_elu_special_cases():
    """ELU: identity for l >= 0; l == u gives the tangent (gamma = 0)."""
    assert oracle.linearize(ELU, 0.0, 2.0) == (1.0, 0.0, 0.0)
    a, b, g = oracle.linearize(ELU, -0.7, -0.7)
    assert a == pytest.approx(math.exp(-0.7), rel=1e-14)
    assert a * -0.7 + b == pytest.approx(math.expm1(-0.7), rel=1e-12)
    assert abs(g) < 1e-14
    # very negative range: f is ~ -1 and flat
    a, b, g = oracle.linearize(ELU, -800.0, -790.0)
    assert abs(a) < 1e-300 and b == pytest.approx(-1.0) and g < 1e-12


def test_sin_wide_and_narrow():
    """sin over >= one period: alpha = 0, beta = 0, gamma = 1. Narrow range
    around an extremum: slope ~ 0, gamma ~ quadratic."""
    a, b, g = oracle.linearize(SIN, -1.0, 1.0 + 2 * math.pi)
    assert a == 0.0 and abs(b) < 1e-15 and g == pytest.approx(1.0)
    a, b, g = oracle.linearize(SIN, math.pi / 2 - 1e-3, math.pi / 2 + 1e-3)
    assert abs(a) < 1e-6 and g < 1e-6
    # on [0, pi/2] sin is concave; the rule's line must bracket it
    a, b, g = oracle.linearize(SIN, 0.0, math.pi / 2)
    hi, lo = max_err(SIN, a, b, 0.0, math.pi / 2)
    assert hi == pytest.approx(g, abs=1e-7) and lo == pytest.approx(-g, abs=1e-7)


@pytest.mark.parametrize("act", [RELU, ELU, SIN, 0])
def test_interval_activation_is_exact_image(act):
    for (l, u) in intervals(31, 200, 4.0):
        lo, hi = oracle.interval_act(act, l, u)
        xs = dense(l, u)
        ys = xs if act == 0 else f_np(act, xs)
        assert lo <= ys.min() + 1e-12 and hi >= ys.max() - 1e-12
        assert lo >= ys.min() - 1e-7 and hi <= ys.max() + 1e-7
