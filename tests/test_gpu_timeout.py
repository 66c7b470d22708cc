"""Failure detection of the tensor-core bound kernel: a bounded device wait
that runs out.

Every mbarrier wait of the tensor-core bound kernel has an iteration budget.
sra_test_tc_stall(spins) switches the kernel's weight copies off and sets
that budget to `spins`, so every wait on a weight stage runs out with no copy
and no MMA in flight. The test checks that the host learns of it
(sra_sync_status returns SRA_ETIMEOUT), that the kernel left before writing
any result, and that the next normal call on the same network is clean and
returns what an undisturbed call returned. No GPU fault is involved.
"""
import ctypes as C

import pytest
import torch

from paper_2202_02444_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sra():
    from paper_2202_02444_gb300 import sra as s
    lib = s.library()
    lib.sra_test_tc_stall.argtypes = [C.c_int32]
    lib.sra_test_tc_stall.restype = C.c_int
    return s


@pytest.mark.parametrize("precision", ["bf16_sound", "bf16"])
def test_wait_runs_out_then_next_call_is_clean(sra, precision):
    lib = sra.library()
    net = sra.Net(wl.make_mlp([128] * 4, "relu", seed=31))
    c, h = wl.make_boxes(1000, seed=7, hw_lo=1 / 256, hw_hi=1 / 16)
    C_, H_ = torch.from_numpy(c).cuda(), torch.from_numpy(h).cuda()
    opts = sra.make_opts(arith="truncate", K=64, precision=precision)
    lo0, hi0, cls0 = sra.bound_boxes(net, C_, H_, opts=opts)
    sra.sync_status(net)

    lo1 = torch.full((1000,), 7.0, device="cuda")
    hi1 = torch.full((1000,), 7.0, device="cuda")
    cls1 = torch.full((1000,), 9, dtype=torch.uint8, device="cuda")
    assert lib.sra_test_tc_stall(64) == sra.OK
    try:
        sra.bound_boxes(net, C_, H_, opts=opts, lo=lo1, hi=hi1, cls=cls1)
        code = lib.sra_sync_status(net.handle, C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert code == sra.ETIMEOUT, lib.sra_last_error()
        assert b"bounded wait" in lib.sra_last_error()
    finally:
        assert lib.sra_test_tc_stall(0) == sra.OK
    # the kernel left before its output layer: nothing was written
    assert torch.all(lo1 == 7.0) and torch.all(hi1 == 7.0) and torch.all(cls1 == 9)
    # the status record was cleared and the context is usable
    sra.sync_status(net)
    lo2, hi2, cls2 = sra.bound_boxes(net, C_, H_, opts=opts)
    sra.sync_status(net)
    assert torch.equal(lo0, lo2) and torch.equal(hi0, hi2) and torch.equal(cls0, cls2)
    net.close()


def test_stall_setting_is_validated(sra):
    lib = sra.library()
    assert lib.sra_test_tc_stall(-1) == sra.EINVAL
    assert lib.sra_test_tc_stall(1 << 21) == sra.EINVAL
    assert lib.sra_test_tc_stall(0) == sra.OK
