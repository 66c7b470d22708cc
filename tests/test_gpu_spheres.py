"""GPU empty-sphere queries (sra_empty_spheres) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_02444_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sra():
    from paper_2202_02444_gb300 import sra as s
    return s


def explained(mlp, p, r_gpu, r_ref, arith, K, band):
    """A mismatch is allowed where the oracle's bound of the box at the larger
    of the two radii lies within band of zero (FP32 may decide it either way)."""
    r = np.maximum(r_gpu, r_ref)
    res = oracle.bound_boxes(mlp, p, np.repeat(r[:, None], 3, 1), arith, K)
    scale = np.abs(res["y0"]) + res["rad"]
    return (np.abs(res["lo"]) <= band * scale) | (np.abs(res["hi"]) <= band * scale)


@pytest.mark.parametrize("which,arith,K", [("small", "fixed", 0), ("elu", "truncate", 8), ("sin", "fixed", 0)])
def test_spheres_vs_oracle(sra, which, arith, K):
    mlp = {"small": wl.net_small_relu(), "elu": wl.make_mlp([64, 64], "elu", seed=4),
           "sin": wl.make_mlp([32, 32], "sin", seed=5)}[which]
    p = np.random.default_rng(7).uniform(-1, 1, (3001, 3)).astype(np.float32)
    net = sra.Net(mlp)
    try:
        rad = sra.empty_spheres(net, torch.from_numpy(p).cuda(), 1.0, 14, arith=arith, K=K).cpu().numpy()
    finally:
        net.close()
    ref = oracle.empty_spheres(mlp, p, 1.0, 14, arith, K)
    mism = rad.astype(np.float64) != ref
    if mism.any():
        ok = explained(mlp, p[mism], rad[mism].astype(np.float64), ref[mism], arith, K, 1e-5)
        assert ok.all(), np.nonzero(mism)[0][~ok][:5]
    assert mism.mean() <= 0.01
    assert (ref > 0).mean() > 0.3


def test_plane_exact_and_fp64(sra):
    nv = np.array([0.3, -0.5, 0.8])
    mlp = wl.make_custom_mlp([3, 1], [], [(nv[None, :], np.array([-0.1]))])
    p = np.random.default_rng(8).uniform(-1, 1, (500, 3)).astype(np.float32)
    net = sra.Net(mlp)
    try:
        r32 = sra.empty_spheres(net, torch.from_numpy(p).cuda(), 1.0, 14).cpu().numpy()
        r64 = sra.empty_spheres(net, torch.from_numpy(p).cuda(), 1.0, 14, precision="fp64").cpu().numpy()
        rre = sra.empty_spheres(net, torch.from_numpy(p).cuda(), 1.0, 14, recheck=True).cpu().numpy()
    finally:
        net.close()
    ref = oracle.empty_spheres(mlp, p, 1.0, 14)
    assert (r64 == ref).mean() >= 0.998
    assert (r32 == ref).mean() >= 0.99 and (rre == ref).mean() >= 0.99


def test_arguments(sra):
    net = sra.Net(wl.net_small_relu())
    try:
        p = torch.zeros((4, 3), device="cuda")
        for kw in (dict(r_max=0.0), dict(levels=0), dict(levels=31)):
            with pytest.raises(sra.SraError) as e:
                sra.empty_spheres(net, p, **kw)
            assert e.value.code == sra.EINVAL
        with pytest.raises(sra.SraError) as e:
            sra.empty_spheres(net, p, precision="bf16")
        assert e.value.code == sra.EUNSUPPORTED
        assert sra.empty_spheres(net, p[:0]).shape[0] == 0
    finally:
        net.close()
