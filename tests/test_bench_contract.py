"""The benchmark's reference arm and its JSON line, on the CPU.

``bench.py --impl reference`` times the float64 oracle on the host cores; it
needs no GPU, so its line is checked here for the keys every benchmark line
carries, on the small chain workload (a few seconds of oracle work). The GPU
arm's line is produced on a GB300 only.
"""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c1",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert k in out, k
    assert out["impl"] == "reference" and out["value"] > 0 and out["higher_is_better"] is True
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["cores"] >= 1
    assert out["cpu_baseline"]["value"] == out["value"]
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in out["config"]


def test_roofline_arithmetic():
    """The roofline entry of the benchmark line: algorithmic work over the
    evolution time against the stated peak, per vector precision."""
    sys.path.insert(0, ROOT)
    import bench as B
    import workloads as W
    models = [W.spin_glass_shard(14, seed=s) for s in range(2)]
    phase = [0.0, 1000.0, 0.0]                          # T_E = 1 s
    clk = {"sm_mhz": 2000.0}
    states = 1e9
    wl = dict(B.WORKLOADS["c3"])
    r = B.roofline(wl, len(models), phase, 3e12, states, clk, 152)
    # double-float: (N b + b + b (b + 1)) multiply-adds x 12 float32 lane operations per state, and
    # b subtractions of w_(k-1) x 8
    ops = 12 * (14 * 4 + 4 + 4 * 5) + 8 * 4
    assert r["bound"] == "alu" and abs(r["achieved"] - states * ops / 1e12) < 1e-9
    assert abs(r["peak"] - 152 * 128 * 2000e6 / 1e12) < 1e-9 and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    wl["prec"] = "fp32"
    r = B.roofline(wl, len(models), phase, 3e12, states, clk, 152)
    assert r["bound"] == "hbm" and abs(r["achieved"] - 3000.0) < 1e-9 and r["unit"] == "GB/s"


def test_sector_levels_rule():
    """Each parity sector is asked for half of n_eigs plus a margin of 1 % (at least 5 levels);
    --sector-share overrides it."""
    sys.path.insert(0, ROOT)
    import bench as B
    assert [B.sector_levels(n) for n in (60, 100, 500, 2000)] == [35, 55, 255, 1020]
    for n in (1, 7, 64, 333, 5000):
        assert n / 2 + 5 <= B.sector_levels(n) <= n / 2 + max(5, 0.01 * n) + 1
    assert B.sector_levels(500, 0.55) == 275
