"""The allocation-free octree round (sra_classify_and_split_noalloc).

Some callers of this library cannot allocate device memory: real-time loops
that forbid allocator calls on the hot path, or hosts that hand over a
pre-partitioned device without an allocator. For them the round keeps its
scratch in a fixed device array. This test calls the variant through the C
ABI and checks that it returns exactly what the allocating entry point
returns, twice in a row (the array keeps the previous call's contents, so the
second call must not depend on them), while every allocation the library
would make is set to fail (a host-side injection: an allocation would turn
into SRA_ENOMEM). The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2202_02444_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sra():
    from paper_2202_02444_gb300 import sra as s
    lib = s.library()
    lib.sra_classify_and_split_noalloc.argtypes = lib.sra_classify_and_split.argtypes
    lib.sra_classify_and_split_noalloc.restype = C.c_int
    return s


def round_via(sra, fn, net, fr, max_level, opts):
    n = fr.shape[0]
    out = torch.full((8 * n, 4), -1, dtype=torch.int16, device="cuda")
    lv = torch.full((n, 4), -1, dtype=torch.int16, device="cuda")
    cnt = torch.zeros(8, dtype=torch.int64, device="cuda")
    rl, rh = (C.c_float * 3)(-1, -1, -1), (C.c_float * 3)(1, 1, 1)
    code = fn(net.handle, C.byref(opts), rl, rh, C.c_void_p(fr.data_ptr()), n, max_level,
              C.c_void_p(out.data_ptr()), 8 * n, C.c_void_p(lv.data_ptr()), n,
              C.c_void_p(cnt.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return code, out, lv, cnt


@pytest.mark.parametrize("recheck", [False, True])
def test_noalloc_round_equals_allocating_round(sra, recheck):
    lib = sra.library()
    net = sra.Net(wl.net_small_relu())
    opts = sra.make_opts(arith="truncate", K=8, recheck=recheck, recheck_band=1e-3)
    for seed, level, max_level in ((9, 5, 6), (10, 6, 6)):  # two calls in a row
        fr = sra.nodes_to_tensor(wl.random_nodes(50000 + seed, level=level, seed=seed))
        c0, o0, l0, n0 = round_via(sra, lib.sra_classify_and_split, net, fr, max_level, opts)
        # any device allocation of the library would now fail with SRA_ENOMEM
        assert lib.sra_test_fail_allocs(1000) == 0
        try:
            c1, o1, l1, n1 = round_via(sra, lib.sra_classify_and_split_noalloc, net, fr, max_level, opts)
        finally:
            lib.sra_test_fail_allocs(0)
        assert c0 == 0 and c1 == 0, lib.sra_last_error()
        assert torch.equal(n0, n1)
        assert torch.equal(o0, o1) and torch.equal(l0, l1)
        assert int(n1[sra.CNT_CHILDREN]) + int(n1[sra.CNT_LEAVES]) > 0
    net.close()


def test_noalloc_rejects_oversized_input(sra):
    lib = sra.library()
    net = sra.Net(wl.net_small_relu())
    opts = sra.make_opts()
    n = 524288 + 1
    fr = torch.zeros((n, 4), dtype=torch.int16, device="cuda")
    code, *_ = round_via(sra, lib.sra_classify_and_split_noalloc, net, fr, 3, opts)
    assert code == sra.EINVAL
    assert b"allocation-free limit" in lib.sra_last_error()
    net.close()


@pytest.mark.parametrize("what", ["bf16_sound", "bf16", "converge", "full_in_device_memory"])
def test_noalloc_rejects_unsupported_options(sra, what):
    lib = sra.library()
    if what == "full_in_device_memory":  # a 128-wide net's full state needs device scratch
        net = sra.Net(wl.make_mlp([128] * 3, "relu", seed=61))
        opts = sra.make_opts(arith="full")
    else:
        net = sra.Net(wl.net_small_relu())
        opts = sra.make_opts(converge=True) if what == "converge" else sra.make_opts(precision=what)
    fr = sra.nodes_to_tensor(wl.random_nodes(64, level=3, seed=3))
    code, *_ = round_via(sra, lib.sra_classify_and_split_noalloc, net, fr, 4, opts)
    assert code == sra.EUNSUPPORTED
    net.close()
