"""The benchmark's reference arm (the FP64 oracle timed on the host cores) on the CPU: one JSON line
with the fields of the benchmark contract, a measured step time that fits inside the process's own
wall clock, and no output from ranks other than 0."""
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ)
    env.update(extra_env or {})
    t0 = time.perf_counter()
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--config", "spin16", "--steps", "2",
                          "--warmup", "1"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return out, time.perf_counter() - t0


def test_reference_arm_prints_one_contract_line():
    out, wall = _run()
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0 and line["higher_is_better"] is True
    # the measured step time of the timed steps fits inside the wall clock of the whole process
    assert line["steps"] * line["ms_per_step"] / 1e3 < wall
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert "spin16" in line["config"]["workload"]


def test_reference_arm_other_ranks_exit_quietly():
    out, _ = _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""
