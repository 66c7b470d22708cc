"""Errors of the device FP32 math functions that the sound activation rules
pad, measured against FP64 (numpy) on many arguments over the ranges the
rules see. The rules assume (sound_rules.cuh):

* sinf, sinpif (the sin rules' extremes): within 4 ulp of the exact value,
  padded by 2^-21 of the result plus the smallest normal float;
* expm1f (the ELU rule's ends): within 2^-22 of the result, plus the smallest
  normal float; expf (its tangent slope): within 2^-21 of the result;
* acosf (the sin rules' critical points): its error lies inside the
  candidates' distance dx, at least 2^-20 (|x| + 8) in radians.

Measured maxima far inside those paddings are evidence for them (CUDA
documents the functions' ulp bounds; this checks the library in use), not a
proof over every float.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

FLT_MIN = np.float64(np.finfo(np.float32).tiny)
N = 1 << 22


@pytest.fixture(scope="module")
def lib():
    from paper_2202_02444_gb300 import sra
    lib = sra.library()
    lib.sra_test_math_f32.argtypes = [C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    lib.sra_test_math_f32.restype = C.c_int
    return lib


def device_eval(lib, fn, x):
    xt = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
    yt = torch.empty_like(xt)
    assert lib.sra_test_math_f32(fn, xt.data_ptr(), xt.numel(), yt.data_ptr(), None) == 0
    torch.cuda.synchronize()
    return yt.cpu().numpy().astype(np.float64)


def args(lo, hi, seed, special=()):
    rng = np.random.default_rng(seed)
    x = rng.uniform(lo, hi, N).astype(np.float32)
    return np.concatenate([x, np.asarray(special, np.float32)])


def quarter_turns(scale, count):
    """Floats next to multiples of pi/2 (radians) or 1/2 (half-turns), where
    sin and cos pass through 0 and +-1."""
    k = np.arange(-count, count + 1, dtype=np.float64) * scale
    base = k.astype(np.float32)
    return np.concatenate([base, np.nextafter(base, np.float32(np.inf)), np.nextafter(base, np.float32(-np.inf))])


@pytest.mark.parametrize("fn,name,ref,lo,hi,special", [
    (0, "sinf", np.sin, -120.0, 120.0, quarter_turns(np.pi / 2, 76)),
    (1, "cosf", np.cos, -120.0, 120.0, quarter_turns(np.pi / 2, 76)),
    (2, "sinpif", lambda x: np.sin(np.pi * x), -200.0, 200.0, quarter_turns(0.5, 400)),
])
def test_sin_family_within_padding(lib, fn, name, ref, lo, hi, special):
    x = args(lo, hi, seed=fn, special=special)
    y = device_eval(lib, fn, x)
    if fn == 2:  # sin(pi x) in FP64: reduce x exactly to [-1/2, 1/2] first, so that integers give 0
        xd = x.astype(np.float64)
        xr = xd - 2.0 * np.round(xd / 2.0)              # [-1, 1], exact
        sgn = np.where(xr < -0.5, -1.0, 1.0)
        xr = np.where(xr > 0.5, 1.0 - xr, np.where(xr < -0.5, 1.0 + xr, xr))  # sin(pi (1 - t)) = sin(pi t)
        exact = sgn * np.sin(np.pi * xr)
    else:
        exact = ref(x.astype(np.float64))
    err = np.abs(y - exact)
    pad = 2.0 ** -21 * np.abs(y) + FLT_MIN
    ulp = np.spacing(np.abs(exact).astype(np.float32)).astype(np.float64)
    print(f"{name}: max error {np.max(err / ulp):.2f} ulp")
    assert np.all(err <= pad), (x[np.argmax(err - pad)], np.max(err - pad))


def test_exp_family_within_padding(lib):
    x = args(-30.0, 0.0, seed=11, special=[0.0, -1e-30, -1e-7, -0.5, -1.0, -20.0, -30.0])
    e = device_eval(lib, 4, x)
    exact = np.expm1(x.astype(np.float64))
    err = np.abs(e - exact)
    assert np.all(err <= 2.0 ** -22 * np.abs(e) + FLT_MIN), np.max(err / (np.abs(e) + FLT_MIN))
    f = device_eval(lib, 5, x)
    exact = np.exp(x.astype(np.float64))
    err = np.abs(f - exact)
    assert np.all(err <= 2.0 ** -21 * np.abs(f) + FLT_MIN), np.max(err / (np.abs(f) + FLT_MIN))


def test_acos_inside_candidate_distance(lib):
    x = args(-1.0, 1.0, seed=12, special=[-1.0, 1.0, np.nextafter(np.float32(1), np.float32(0)),
                                           np.nextafter(np.float32(-1), np.float32(0)), 0.0])
    y = device_eval(lib, 3, x)
    err = np.abs(y - np.arccos(x.astype(np.float64)))
    print(f"acosf: max error {err.max():.2e} rad")
    assert err.max() <= 2.0 ** -20 * 8


def test_bad_arguments(lib):
    assert lib.sra_test_math_f32(7, None, 0, None, None) != 0
    assert lib.sra_test_math_f32(0, None, -1, None, None) != 0
    assert lib.sra_test_math_f32(0, None, 0, None, None) == 0
