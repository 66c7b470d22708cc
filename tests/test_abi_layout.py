"""CPU check that the ctypes mirrors of the public structs in the Python
binding have the C layout of include/sra.h: a small C program compiled with
the host compiler prints sizeof and every field's offsetof, and each ctypes
Structure must agree field by field. A field added on one side only, or
reordered, fails here before it can corrupt a call."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def c_layout(tmp_path, structs):
    """{struct: (sizeof, {field: offset})} from the host C compiler."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "sra.h"', "int main(void) {"]
    for name, fields in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f in fields:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    res = {name: [None, {}] for name in structs}
    for line in out.splitlines():
        name, field, value = line.split()
        if field == "size":
            res[name][0] = int(value)
        else:
            res[name][1][field] = int(value)
    return res


def test_ctypes_structs_match_the_header(tmp_path):
    from paper_2202_02444_gb300 import sra
    mirrors = {"sra_opts": sra.Opts, "sra_mlp_desc": sra.MlpDesc, "sra_batch_seg": sra.BatchSeg,
               "sra_request": sra.Request, "sra_serve_cfg": sra.ServeCfg}
    structs = {name: [f[0] for f in cls._fields_] for name, cls in mirrors.items()}
    layout = c_layout(tmp_path, structs)
    for name, cls in mirrors.items():
        size, offsets = layout[name]
        assert C.sizeof(cls) == size, (name, C.sizeof(cls), size)
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == offsets[field], (name, field)


def test_node_record_is_eight_bytes(tmp_path):
    from paper_2202_02444_gb300 import sra
    layout = c_layout(tmp_path, {"sra_node": ["ix", "iy", "iz", "level"]})
    size, offsets = layout["sra_node"]
    assert size == sra.NODE_DTYPE.itemsize == 8
    assert [offsets[f] for f in ("ix", "iy", "iz", "level")] == [sra.NODE_DTYPE.fields[f][1]
                                                                for f in ("ix", "iy", "iz", "level")]
