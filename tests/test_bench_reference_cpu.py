"""The benchmark's reference arm (the CPU oracle over all host cores) runs without a GPU
and prints one JSON line with the contract's keys; its per-step sample shrinks so that
a large --steps still finishes quickly."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args, n=20000):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--n", str(n), "--nq", "400", *args],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    j = _run("--steps", "3", "--warmup", "1")
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert key in j, key
    assert j["impl"] == "reference" and j["steps"] == 3 and j["value"] > 0
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == j["value"]
    assert j["e2e"]["h2d_bytes_per_step"] == 0 and j["e2e"]["value"] == j["value"]


def test_reference_arm_bounds_its_run_time():
    # (each step also pays a thread-pool dispatch of about 2 ms, so the step count is kept
    # where that floor stays below the budget)
    j = _run("--steps", "2000", "--warmup", "3", "--ref-seconds", "4")
    assert j["steps"] == 2000
    # about --ref-seconds of oracle work in all, whatever the step count
    assert j["ms_per_step"] * j["steps"] / 1000.0 < 20
    # the value is an all-cores rate in every regime
    assert j["cpu_baseline"]["cores"] == (os.cpu_count() or 1)


def test_reference_arm_time_bound_at_a_larger_object_count():
    # one query per thread over all 200,000 objects is longer than a step's budget, so
    # every thread scans a prefix sized to it; all cores stay in use
    j = _run("--steps", "1500", "--warmup", "3", "--ref-seconds", "3", n=200000)
    assert j["steps"] == 1500
    assert j["ms_per_step"] * j["steps"] / 1000.0 < 15
    assert j["cpu_baseline"]["cores"] == (os.cpu_count() or 1)
    assert "rate scaled by" in j["cpu_baseline"]["sample"]
