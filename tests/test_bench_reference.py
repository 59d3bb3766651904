"""bench.py's reference arm (the FP64 CPU oracle timed on bounded samples of
the workload): the one JSON line of the timing contract, on the smallest
workload, and the quiet exit of every rank but 0 under a multi-rank launch."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e")


def run_reference(extra_env):
    env = dict(os.environ)
    env.update(extra_env)
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--config", "1", "--steps", "2", "--warmup", "1",
           "--ref-window", "32"]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)


def test_reference_arm_prints_one_contract_line():
    r = run_reference({})
    assert r.returncode == 0, r.stderr
    lines = [line for line in r.stdout.splitlines() if line.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in KEYS:
        assert k in d, k
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert (d["steps"], d["warmup"], d["n_gpus"]) == (2, 1, 1)
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"].startswith("c1_")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work():
    r = run_reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
