"""Independent numpy forward pass of an MLP (test helper, fp64).

Written directly from the network definition (linear layers, activations,
positional encoding [x, per octave sin(2^k pi x), cos(2^k pi x)]) so that
brute-force soundness checks do not depend on the oracle's own evaluator.
"""
import numpy as np


def forward(mlp, x):
    x = np.asarray(x, np.float64).reshape(-1, 3)
    h = x
    if mlp.pe_octaves:
        feats = [x]
        for k in range(mlp.pe_octaves):
            z = (2.0 ** k) * np.pi * x
            feats.append(np.sin(z))
            feats.append(np.cos(z))
        h = np.concatenate(feats, axis=1)
    for l in range(mlp.n_layers):
        W, b = mlp.layer(l)
        h = h @ W.astype(np.float64).T + b.astype(np.float64)
        if l < mlp.n_layers - 1:
            a = mlp.acts[l]
            if a == 1:
                h = np.maximum(h, 0.0)
            elif a == 2:
                h = np.where(h > 0, h, np.expm1(np.minimum(h, 0.0)))
            elif a == 3:
                h = np.sin(h)
    return h[:, 0]


def box_samples(center, halfw, n_grid=4, n_rand=64, seed=0):
    """Grid (n_grid^3, incl. corners) plus random points inside a box."""
    rng = np.random.default_rng(seed)
    t = np.linspace(-1.0, 1.0, n_grid)
    g = np.stack(np.meshgrid(t, t, t, indexing="ij"), -1).reshape(-1, 3)
    r = rng.uniform(-1.0, 1.0, size=(n_rand, 3))
    e = np.concatenate([g, r])
    return np.asarray(center)[None, :] + e * np.asarray(halfw)[None, :]
