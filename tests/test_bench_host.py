"""Host-side parts of the benchmark that need no GPU: the oracle's bounded
CPU sample (its repeat bound and reported threads) and the reference arm's
JSON line, which times the oracle on the full 257x257, N = 256 workload."""
import json
import os
import subprocess
import sys

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_sample_repeats_and_threads():
    import bench
    prob = W.config_plain_fp64()
    s = bench.oracle_sample(prob, 10, min_seconds=1e9, max_repeats=3)
    assert "3 time(s)" in s["sample"]
    assert s["value"] > 0 and s["extrapolated_solve_s"] > 0
    assert 1 <= s["cores"] <= max(1, s["cores_visible"]) + 1
    one = bench.oracle_sample(prob, 10)
    assert "1 time(s)" in one["sample"]
    # more outer iterations, longer extrapolated solve
    assert bench.oracle_sample(prob, 1000)["extrapolated_solve_s"] > one["extrapolated_solve_s"]


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=900,
                         cwd=ROOT, env=dict(os.environ, RANK="0"))
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unit"] == "DOF/s" and line["higher_is_better"] is True
    assert line["config"]["workload"] == "square257_N256"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "DOF/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    # value = space-time DOFs / extrapolated solve time
    assert abs(line["value"] * line["ms_per_step"] / 1e3 - 65025 * 256) < 1e-6 * 65025 * 256


def test_reference_arm_other_ranks_exit_without_work():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=300,
                         cwd=ROOT, env=dict(os.environ, RANK="1"))
    assert out.returncode == 0 and out.stdout.strip() == ""
