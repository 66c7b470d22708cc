"""CPU checks of the C ABI: the library loads and exports every function the
public header declares (no compute calls; no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")
LIB = os.path.join(ROOT, "paper_2202_02444_gb300", "libsra.so")


def declared_functions():
    names = []
    for h in sorted(os.listdir(HEADER_DIR)):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(sra_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2202_02444_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sra_load_mlp", "sra_free_mlp", "sra_bound_boxes", "sra_classify_and_split",
                 "sra_cast_rays", "sra_extract_leaves", "sra_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_exports_are_c_linkage():
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (sra_[a-z0-9_]+)\b", out))
    assert set(declared_functions()) <= exported


def test_default_opts_without_gpu(lib):
    from paper_2202_02444_gb300 import sra
    o = sra.make_opts()
    assert o.arith == 1 and abs(o.delta - 1e-3) < 1e-9 and o.eta_plus == 1.5
    assert o.safety == pytest.approx(0.98) and o.max_iters == 1 << 20
