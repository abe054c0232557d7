"""bench.py's reference arm on CPU: the JSON line it prints (the oracle timed on the host,
the same metric and unit as the CUDA arm) and the silent exit of ranks other than 0."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra, *args):
    env = dict(os.environ)
    env.update(env_extra)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    return r.stdout


def test_reference_line_contract():
    out = _run({}, "--workload", "1", "--steps", "2", "--warmup", "1")
    lines = [ln for ln in out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "PGD-TO optimizer steps/s" and d["unit"] == "steps/s"
    assert d["higher_is_better"] is True and d["value"] > 0.0
    assert d["warmup"] >= 3  # at least three untimed warm-up steps, whatever was asked
    assert d["steps"] >= 1 and abs(d["ms_per_step"] - 1e3 / d["value"]) <= 1e-6 * d["ms_per_step"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"]


def test_reference_other_ranks_print_nothing():
    out = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--workload", "1", "--steps", "1")
    assert out.strip() == ""


def test_roofline_arithmetic():
    """The byte counts and roofline fractions the bench line reports, against values worked
    out by hand for workload 3 (n = 7,077,888, one coefficient per variable, 3 passes)."""
    sys.path.insert(0, ROOT)
    import bench
    n = 7077888
    # 16 (phase A) + 24 (phase B: 20 + 4) + 4 * 2 * 3 (passes) + 16 (phase D: 12 + 4) = 80 bytes
    assert bench.algorithmic_bytes(n, 1, 3) == 80 * n
    # x, x_prev, g, g_prev, d_prev, a read once (24) and d, x_new written once (8)
    assert bench.compulsory_bytes(n, 1) == 32 * n
    assert bench.pass_bytes(n, 1) == 8 * n
    # coupled rows: four dense coefficient rows per variable
    assert bench.compulsory_bytes(n, 4) == (4 * 9 + 8) * n and bench.pass_bytes(n, 4) == 20 * n
    step_s = 250e-6
    r = bench.roofline(n, 1, 3, step_s, 6800.0, 6600.0, None, "k")
    assert abs(r["achieved"] - 80 * n / step_s / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6800.0) < 1e-12
    # the passes fit L2 (56.6 MB): they count at the L2 rate, the compulsory bytes at HBM's
    floor = 32 * n / 6800e9 + 3 * 8 * n / 6600e9
    assert abs(r["split_floor_us"] - 1e6 * floor) < 1e-9
    assert abs(r["frac_split"] - floor / step_s) < 1e-12
    assert abs(r["frac_compulsory"] - 32 * n / step_s / 1e9 / 6800.0) < 1e-12
    # a pass larger than L2 counts at the HBM rate
    big = 40_000_000
    r2 = bench.roofline(big, 1, 2, step_s, 6800.0, 6600.0, None, "k")
    assert abs(r2["split_floor_us"] - 1e6 * (32 * big + 2 * 8 * big) / 6800e9) < 1e-9
