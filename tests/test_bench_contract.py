"""The benchmark's reference arm (the FP64 oracle timed on the host cores) prints one JSON line with
the fields the benchmark contract asks for; it runs without a GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "0"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["steps"] == 2 and d["n_gpus"] == 1 and d["value"] > 0
    assert d["higher_is_better"] is False and d["unit"] == "s/map"
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_under_two_ranks_prints_on_rank_zero_only():
    outs = {}
    for rank in (0, 1):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank))
        out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                              "--steps", "1", "--warmup", "0"], capture_output=True, text=True, cwd=ROOT, env=env,
                             timeout=600)
        assert out.returncode == 0, out.stderr[-2000:]
        outs[rank] = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert outs[1] == [] and len(outs[0]) == 1
    d = json.loads(outs[0][0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
