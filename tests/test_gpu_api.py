"""Error handling of the C ABI on a GPU host: bad arguments return status
codes (nothing traps), sra_last_error explains them."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2202_02444_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sra():
    from paper_2202_02444_gb300 import sra as s
    return s


def test_load_rejects_bad_shapes(sra):
    lib = sra.library()
    w = np.array([3, 8, 2], np.int32)  # last width must be 1
    a = np.array([1], np.int32)
    p = np.zeros(3 * 8 + 8 + 8 * 2 + 2, np.float32)
    d = sra.MlpDesc(2, w.ctypes.data_as(C.POINTER(C.c_int32)), a.ctypes.data_as(C.POINTER(C.c_int32)),
                    p.ctypes.data_as(C.POINTER(C.c_float)), 0)
    h = C.c_void_p()
    assert lib.sra_load_mlp(C.byref(d), C.byref(h)) == sra.EINVAL
    assert b"widths" in lib.sra_last_error()
    w2 = np.array([3, 1024, 1], np.int32)
    d.widths = w2.ctypes.data_as(C.POINTER(C.c_int32))
    assert lib.sra_load_mlp(C.byref(d), C.byref(h)) == sra.EUNSUPPORTED


def test_bad_options_and_sizes(sra):
    mlp = wl.net_small_relu()
    net = sra.Net(mlp)
    c = torch.zeros((4, 3), device="cuda")
    with pytest.raises(sra.SraError) as e:
        sra.bound_boxes(net, c, c, arith="truncate", K=0)
    assert e.value.code == sra.EINVAL
    with pytest.raises(sra.SraError) as e:
        sra.bound_boxes(net, c, c, arith="truncate", K=4096)
    assert e.value.code == sra.EUNSUPPORTED
    with pytest.raises(sra.SraError) as e:
        sra.cast_rays(net, c, c, delta=0.0)
    assert e.value.code == sra.EINVAL
    fr = torch.zeros((1, 4), dtype=torch.int16, device="cuda")
    with pytest.raises(sra.SraError) as e:
        sra.classify_and_split(net, fr, max_level=40)
    assert e.value.code == sra.EINVAL
    lib = sra.library()
    o = sra.make_opts()
    assert lib.sra_bound_boxes(net.handle, C.byref(o), None, None, 4, None, None, None, None) == sra.EINVAL
    assert lib.sra_bound_boxes(net.handle, C.byref(o), None, None, -1, None, None, None, None) == sra.EINVAL
    assert lib.sra_bound_boxes(None, C.byref(o), None, None, 4, None, None, None, None) == sra.EINVAL
    net.close()


def test_leaf_capacity_status(sra):
    mlp = wl.net_small_relu()
    net = sra.Net(mlp)
    lib = sra.library()
    o = sra.make_opts()
    buf = torch.empty((10, 4), dtype=torch.int16, device="cuda")
    nl = C.c_int64(0)
    code = lib.sra_extract_leaves(net.handle, C.byref(o), (C.c_float * 3)(-1, -1, -1),
                                  (C.c_float * 3)(1, 1, 1), 5, C.c_void_p(buf.data_ptr()), 10,
                                  C.byref(nl), None, None)
    torch.cuda.synchronize()
    assert code == sra.ECAPACITY and nl.value > 10
    net.close()


def test_injected_allocation_failures(sra):
    """An injected allocation failure (host-side, sra_test_fail_allocs) makes
    the call that needed the allocation return SRA_ENOMEM; the same call then
    succeeds and returns what an undisturbed call returns."""
    lib = sra.library()
    lib.sra_test_fail_allocs.argtypes = [C.c_int32]
    lib.sra_test_fail_allocs.restype = C.c_int
    assert lib.sra_test_fail_allocs(-1) == sra.EINVAL
    mlp = wl.net_small_relu()
    try:
        assert lib.sra_test_fail_allocs(1) == sra.OK
        with pytest.raises(sra.SraError) as e:
            sra.Net(mlp)
        assert e.value.code == sra.ENOMEM and b"injected" in lib.sra_last_error()
        net = sra.Net(mlp)
        c, h = wl.make_boxes(300, seed=4)
        C_, H_ = torch.from_numpy(c).cuda(), torch.from_numpy(h).cuda()
        o, d = wl.sphere_rays(24, seed=5, radius=2.0)
        O_, D_ = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
        root = sra.nodes_to_tensor(wl.root_node())
        calls = {
            "boxes (FP64 re-check scratch)": lambda: sra.bound_boxes(net, C_, H_, arith="fixed", recheck=True,
                                                                     recheck_band=1e-2)[0],
            "octree round": lambda: sra.classify_and_split(net, root, 4, arith="fixed")[2],
            "rays": lambda: sra.cast_rays(net, O_, D_, arith="fixed", delta=1e-3)[0],
        }
        for name, call in calls.items():
            ref = call().cpu().numpy()
            assert lib.sra_test_fail_allocs(1) == sra.OK
            with pytest.raises(sra.SraError) as e:
                call()
            assert e.value.code == sra.ENOMEM, name
            again = call().cpu().numpy()
            assert np.array_equal(again.view(np.uint8), ref.view(np.uint8)), name
        net.close()
    finally:
        lib.sra_test_fail_allocs(0)
