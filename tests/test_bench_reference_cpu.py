"""The benchmark's reference arm (the CPU oracle over all host cores) runs without a GPU
and prints one JSON line with the contract's keys; its per-step sample shrinks so that
a large --steps still finishes quickly."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--n", "20000", "--nq", "400", *args],
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
    j = _run("--steps", "20000", "--warmup", "3", "--ref-seconds", "4")
    assert j["steps"] == 20000
    # about --ref-seconds of oracle work in all, whatever the step count
    assert j["ms_per_step"] * j["steps"] / 1000.0 < 20
