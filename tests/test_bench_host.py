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
    # value = space-time DOFs / extrapolated solve time, labelled as an
    # extrapolation; ms_per_step is the sample's own wall time
    ext = line["config"]["extrapolated_solve_s"]
    assert abs(line["value"] * ext - 65025 * 256) < 1e-6 * 65025 * 256
    assert line["cpu_baseline"]["extrapolated"] is True and "not an oracle measurement" in \
        line["config"]["iterations_source"]
    assert line["ms_per_step"] / 1e3 == line["config"]["sample_wall_s_per_step"] * 1e3 / 1e3
    assert line["ms_per_step"] / 1e3 < 120.0


def test_oracle_to_tolerance_is_a_measured_solve():
    """cpu_baseline: the oracle's fixed point timed from U = 0 to the stopping
    rule on the 33x33, N = 32 workload (its own iteration count)."""
    import bench
    s = bench.oracle_to_tolerance()
    assert s["converged"] and s["outer_iterations"] > 100
    assert s["workload"] == "square33_N32" and s["space_time_dofs"] == 961 * 32
    assert abs(s["value"] * s["solve_s"] - 961 * 32) < 1e-6 * 961 * 32
    assert 1 <= s["cores"] <= max(1, s["cores_visible"]) + 1


def test_reference_arm_other_ranks_exit_without_work():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=300,
                         cwd=ROOT, env=dict(os.environ, RANK="1"))
    assert out.returncode == 0 and out.stdout.strip() == ""
