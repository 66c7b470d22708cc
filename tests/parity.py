"""Comparison helpers for GPU-vs-oracle parity tests.

Tolerances (stated once, used by every parity test):
  * FP32 centers and radii: |d| <= 1e-5 * (|c_ref| + r_ref), the relative
    tolerance the FP32 form is held to; c cancels, so the scale includes r.
  * FP64 on the GPU: |d| <= 1e-9 * (|c_ref| + r_ref) (summation order and
    FMA differ from the oracle's plain loops).
  * Classes: identical, except where the oracle's lo or hi lies within
    `zero_band` * (1 + |c_ref| + r_ref) of zero.
  * Affine-truncate: a box whose oracle selection had a relative score gap
    below 1e-4 (the last kept vs the first dropped column) may keep another,
    equally valid column set in FP32; such boxes are exempt and counted.
"""
import numpy as np

FP32_REL = 1e-5
FP64_REL = 1e-9
TIE_GAP = 1e-4


def compare_bounds(lo, hi, cls, ref, rel=FP32_REL, zero_band=1e-6, tie_gap=TIE_GAP):
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    cls = np.asarray(cls)
    c_g, r_g = 0.5 * (lo + hi), 0.5 * (hi - lo)
    scale = np.abs(ref["y0"]) + ref["rad"]
    tie = ref.get("sel_gap", np.full(len(lo), np.inf)) < tie_gap
    # float32 storage of lo/hi adds up to one ulp of |lo| + |hi|
    store = 2.0 ** -23 * (np.abs(ref["lo"]) + np.abs(ref["hi"]))
    bad_c = (np.abs(c_g - ref["y0"]) > rel * scale + store) & ~tie
    bad_r = (np.abs(r_g - ref["rad"]) > rel * scale + store) & ~tie
    near = np.minimum(np.abs(ref["lo"]), np.abs(ref["hi"])) <= zero_band * (1.0 + scale)
    bad_cls = (cls != ref["cls"]) & ~near & ~tie
    return {
        "n": len(lo), "bad_center": int(bad_c.sum()), "bad_radius": int(bad_r.sum()),
        "bad_class": int(bad_cls.sum()), "near_zero": int(near.sum()), "ties": int(tie.sum()),
        "max_rel_c": float(np.max(np.abs(c_g - ref["y0"]) / np.maximum(scale, 1e-300))),
        "max_rel_r": float(np.max(np.abs(r_g - ref["rad"]) / np.maximum(scale, 1e-300))),
        "idx_bad": np.nonzero(bad_c | bad_r | bad_cls)[0][:10].tolist(),
    }


def assert_parity(rep, max_tie_frac=0.05):
    assert rep["bad_center"] == 0 and rep["bad_radius"] == 0 and rep["bad_class"] == 0, rep
    assert rep["ties"] <= max_tie_frac * rep["n"], rep


def soundness_violations(lo, hi, samples_f, tol_rel=0.0):
    """Count boxes whose sampled values leave [lo, hi] (beyond tol_rel*scale)."""
    lo = np.asarray(lo, np.float64)[:, None]
    hi = np.asarray(hi, np.float64)[:, None]
    scale = np.abs(lo) + np.abs(hi)
    out = (samples_f < lo - tol_rel * scale) | (samples_f > hi + tol_rel * scale)
    return int(out.any(axis=1).sum())
