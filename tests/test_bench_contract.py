"""The JSON line of bench.py's reference arm (the FP64 oracle timed on the
host cores) carries the keys the measurement contract asks for.  The GPU
arm's line is produced on a GPU only; its keys are built by the same
helpers and checked there by running bench.py."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    _check_reference_line(out, "batched_inclusion_256_literal_mixed")


def test_reference_arm_json_line_single_inclusion():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload",
                          "inclusion", "--steps", "1", "--warmup", "0"], cwd=ROOT,
                         capture_output=True, text=True, timeout=300)
    _check_reference_line(out, "inclusion_osmpm_2d_fp64")


def _check_reference_line(out, workload):
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["config"]["workload"].startswith(workload)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_clock_rows_summary():
    """The clocks object of the bench line: median SM clock under load, the
    maximum clock, and every throttle reason seen active (a run with a
    hardware or thermal slowdown is rejected; sw_power_cap is noted)."""
    sys.path.insert(0, ROOT)
    import bench
    rows = ["0, 2070, 2070, 850.10, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 1950, 2070, 1390.52, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1120.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",
            "garbage"]
    c = bench.parse_clock_rows(rows)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 4}
    hot = bench.parse_clock_rows(["0, 1500, 2070, 1300, 0x48, Active, Not Active, Active, Not Active"])
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and hot["sm_mhz"] == 1500.0
    assert bench.parse_clock_rows([]) is None


def test_hertz_profile_fit_recovers_a_semi_ellipse():
    """The Hertz study's fit returns the half-width and peak of an exact
    semi-elliptic profile, and the closed form satisfies F = pi b p_max / 2
    (the load of a semi-ellipse)."""
    import numpy as np
    import bench
    xc = np.arange(1.75, 2.25, 1 / 256) + 0.5 / 256
    F = 15000.0
    h0 = bench.hertz_profile(np.zeros_like(xc), xc, F)
    b, p0 = h0["b_hertz"], h0["p_max_hertz"]
    assert abs(np.pi * b * p0 / 2 - F) <= 1e-9 * F
    p = 0.8 * p0 * np.sqrt(np.clip(1 - ((xc - 2) / (1.2 * b)) ** 2, 0, None))
    h = bench.hertz_profile(p, xc, F)
    assert abs(h["b_fit"] / (1.2 * b) - 1) < 0.01
    assert abs(h["p_max_fit"] / (0.8 * p0) - 1) < 0.01
