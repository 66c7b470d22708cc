"""CPU check of bench.py's reference arm (the FP64 oracle timed on the host
cores): it prints one JSON line with the native arm's metric and the keys the
benchmark contract asks for, and a rank other than 0 exits 0 without work."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(env_extra, *args):
    env = dict(os.environ, **env_extra)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
        if k not in env_extra:
            env.pop(k, None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout


def test_reference_line_follows_the_contract():
    out = run({}, "--steps", "2", "--warmup", "1", "--ref-sample", "16")
    line = json.loads(out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == "box-bound evals/s" and line["unit"] == "box-bound evals/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 1 and line["ms_per_step"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert "workload" in line["config"]


def test_other_ranks_do_no_work():
    out = run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--steps", "1", "--warmup", "0")
    assert out.strip() == ""


def test_gpus_flag_starts_one_rank_per_gpu():
    """`--gpus 2` without a launcher re-runs the script under
    torch.distributed.run with two ranks; rank 0 alone prints the line and
    reports both ranks."""
    out = run({}, "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-sample", "4")
    lines = [l for l in out.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
