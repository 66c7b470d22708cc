"""The debug build (-DSRA_DEBUG_BOUNDS) of the library: the tensor-core
kernels check their data-dependent indices (kept-symbol list, one-hot rows,
operand write-back rows, re-check lists) before use and record a failed check
in the status word instead of faulting. This test builds that variant in a
temporary copy of the package and runs BF16-sound bounds with the FP64
re-check and BF16 rays with the re-check on it, in a subprocess: no check may
fire (sra_sync_status stays OK) and the results equal the release build's."""
import os
import shutil
import subprocess
import sys
import textwrap

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu

SCRIPT = textwrap.dedent("""
    import sys
    import numpy as np
    import torch
    sys.path.insert(0, sys.argv[1])
    from paper_2202_02444_gb300 import build as B
    B.build(extra=sys.argv[3:])
    from paper_2202_02444_gb300 import sra, workloads as wl
    out = {}
    net = sra.Net(wl.make_mlp([128] * 4, "relu", seed=31))
    c, h = wl.make_boxes(301, seed=2, hw_lo=1 / 512, hw_hi=1 / 16)
    lo, hi, cls = sra.bound_boxes(net, torch.from_numpy(c).cuda(), torch.from_numpy(h).cuda(), arith="truncate",
                                  K=64, precision="bf16_sound", recheck=True, recheck_band=1e-2)
    sra.sync_status(net)
    out["lo"], out["hi"], out["cls"] = lo.cpu().numpy(), hi.cpu().numpy(), cls.cpu().numpy()
    net.close()
    net = sra.Net(wl.make_mlp([128] * 4, "elu", seed=35, pe_octaves=3))
    o, d = wl.sphere_rays(96, seed=8, radius=2.0)
    t, it = sra.cast_rays(net, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), arith="fixed", delta=1e-3,
                          max_iters=2000, precision="bf16", recheck=True, recheck_band=3e-2)
    sra.sync_status(net)
    out["t"], out["it"] = t.cpu().numpy(), it.cpu().numpy()
    net.close()
    np.savez(sys.argv[2], **out)
""")


def run_variant(tmp_path, name, flags):
    root = tmp_path / name
    os.makedirs(root)
    shutil.copytree(os.path.join(ROOT, "paper_2202_02444_gb300"), root / "paper_2202_02444_gb300",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "include"), root / "include")
    script = tmp_path / "run.py"
    script.write_text(SCRIPT)
    res = tmp_path / f"{name}.npz"
    r = subprocess.run([sys.executable, str(script), str(root), str(res), *flags], capture_output=True, text=True,
                       cwd=str(tmp_path))
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(res)


def test_debug_index_checks_stay_silent(tmp_path):
    dbg = run_variant(tmp_path, "debug", ["-DSRA_DEBUG_BOUNDS"])
    rel = run_variant(tmp_path, "release", [])
    for k in rel.files:
        assert np.array_equal(dbg[k].view(np.uint8), rel[k].view(np.uint8)), k
