"""Tensor-core building blocks (sra_selftest_tc_gemm): TMA-loaded swizzled
K-major BF16 weight tiles, thread-written operand tiles, tcgen05.mma into TMEM
and tcgen05.ld, checked against an FP64 product of the same BF16 values."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2202_02444_gb300 import sra
    L = sra.library()
    L.sra_selftest_tc_gemm.argtypes = [C.c_void_p] * 5
    L.sra_selftest_tc_gemm.restype = C.c_int
    return L


@pytest.mark.parametrize("seed", [0, 1])
def test_tc_gemm_matches_fp64(lib, seed):
    g = torch.Generator().manual_seed(seed)
    W = torch.randn(256, 256, generator=g).to(torch.bfloat16)
    X = torch.randn(144, 256, generator=g).to(torch.bfloat16)
    Wd, Xd = W.cuda(), X.cuda()
    D = torch.full((256, 144), float("nan"), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    code = lib.sra_selftest_tc_gemm(C.c_void_p(Wd.data_ptr()), C.c_void_p(Xd.data_ptr()),
                                    C.c_void_p(D.data_ptr()), C.c_void_p(st.data_ptr()),
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert code == 0 and int(st) == 0
    ref = W.double() @ X.double().T
    mag = W.double().abs() @ X.double().abs().T
    err = (D.cpu().double() - ref).abs()
    assert torch.all(err <= 1e-5 * mag + 1e-6), float((err / (mag + 1e-30)).max())
