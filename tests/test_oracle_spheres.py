"""Pins of the empty-sphere oracle (Sec. 4.4): the closed form on a plane
(affine bounds of a linear function are exact) and soundness on random
networks by dense sampling inside every returned ball."""
import numpy as np

import oracle
from paper_2202_02444_gb300 import workloads as wl


def test_plane_closed_form():
    nv = np.array([0.3, -0.5, 0.8])
    d = 0.1
    mlp = wl.make_custom_mlp([3, 1], [], [(nv[None, :], np.array([-d]))])
    n32 = nv.astype(np.float32).astype(np.float64)
    d32 = float(np.float32(d))
    p = np.random.default_rng(1).uniform(-1, 1, (300, 3)).astype(np.float32).astype(np.float64)
    got = oracle.empty_spheres(mlp, p, 1.0, 14, "fixed")
    f = np.abs(p @ n32 - d32)
    L1 = np.abs(n32).sum()
    want = np.zeros(len(p))
    for i in range(len(p)):
        for k in range(14):
            r = 2.0 ** -k
            if r * L1 < f[i]:  # the box range is f(p) +- r |n|_1, decided strictly
                want[i] = r
                break
    assert np.array_equal(got, want)
    assert (want > 0).mean() > 0.9


def test_balls_miss_the_surface():
    rng = np.random.default_rng(2)
    for mlp, arith, K in ((wl.net_small_relu(), "fixed", 0),
                          (wl.make_mlp([32, 32], "elu", seed=3), "truncate", 8)):
        p = rng.uniform(-1, 1, (60, 3))
        rad = oracle.empty_spheres(mlp, p, 1.0, 12, arith, K)
        assert (rad > 0).mean() > 0.5
        f0 = oracle.evaluate(mlp, p)
        for i in np.nonzero(rad > 0)[0]:
            u = rng.normal(size=(400, 3))
            u *= (rng.uniform(0, 1, (400, 1)) ** (1 / 3)) / np.linalg.norm(u, axis=1, keepdims=True)
            f = oracle.evaluate(mlp, p[i] + rad[i] * u)
            assert (np.sign(f) == np.sign(f0[i])).all()
