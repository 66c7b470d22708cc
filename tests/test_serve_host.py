"""CPU checks of sra_serve's argument validation: every rejected trace is
refused before any device work (the network handles are never used)."""
import ctypes as C
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2202_02444_gb300", "libsra.so")


class Request(C.Structure):
    _fields_ = [("kind", C.c_int32), ("net", C.c_int32), ("form", C.c_int32), ("depth", C.c_int32),
                ("arrival", C.c_double), ("n", C.c_int64),
                ("a", C.c_void_p), ("b", C.c_void_p), ("lo", C.c_void_p), ("hi", C.c_void_p),
                ("iters", C.c_void_p), ("cls", C.c_void_p), ("leaves", C.c_void_p),
                ("cap", C.c_int64), ("n_out", C.c_int64), ("status", C.c_int32),
                ("slot", C.c_int32), ("levels", C.c_int32), ("pad", C.c_int32),
                ("t_admit", C.c_double), ("t_done", C.c_double)]


class Cfg(C.Structure):
    _fields_ = [("slots", C.c_int32), ("realtime", C.c_int32), ("frontier_bytes", C.c_int64)]


class Opts(C.Structure):  # layout of sra_opts; contents unused by these cases
    _fields_ = [("raw", C.c_byte * 256)]


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2202_02444_gb300 import build
        build.build()
    L = C.CDLL(LIB)
    L.sra_serve.restype = C.c_int
    L.sra_serve.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.c_void_p, C.c_int32,
                            C.POINTER(Cfg), C.POINTER(Request), C.c_int64]
    L.sra_last_error.restype = C.c_char_p
    return L


def run(lib, reqs, slots=2, n_forms=1, nets=(8,)):
    handles = (C.c_void_p * len(nets))(*nets)
    arr = (Request * max(1, len(reqs)))(*reqs)
    forms = (Opts * n_forms)()
    cfg = Cfg(slots, 0, 1 << 20)
    code = lib.sra_serve(handles, len(nets), C.cast(forms, C.c_void_p), n_forms, C.byref(cfg), arr,
                         len(reqs))
    return code, lib.sra_last_error().decode()


def test_bad_slot_count(lib):
    assert run(lib, [Request(kind=0, net=0, form=0)], slots=0)[0] == 1
    assert run(lib, [Request(kind=0, net=0, form=0)], slots=65)[0] == 1


def test_indices_out_of_range(lib):
    code, msg = run(lib, [Request(kind=0, net=1, form=0)])
    assert code == 1 and "out of range" in msg
    code, msg = run(lib, [Request(kind=0, net=0, form=3)])
    assert code == 1 and "out of range" in msg
    code, msg = run(lib, [Request(kind=7, net=0, form=0)])
    assert code == 1 and "kind" in msg


def test_arrivals_must_not_decrease(lib):
    code, msg = run(lib, [Request(kind=1, net=0, form=0, arrival=1.0),
                          Request(kind=1, net=0, form=0, arrival=0.5)])
    assert code == 1 and "arrives before" in msg


def test_leaf_job_arguments(lib):
    code, msg = run(lib, [Request(kind=2, net=0, form=0, depth=3, cap=0, leaves=16)])
    assert code == 1 and "leaf job" in msg
    code, msg = run(lib, [Request(kind=2, net=0, form=0, depth=16, cap=8, leaves=16)])
    assert code == 1 and "leaf job" in msg


def test_null_network(lib):
    code, msg = run(lib, [Request(kind=0, net=0, form=0)], nets=(None,))
    assert code == 1 and "NULL" in msg
