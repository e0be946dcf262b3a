"""Host-side checks of bench.py (no GPU): the JSON line of the reference arm carries the keys the
benchmark contract fixes, and the algorithmic byte model scales as its definition says."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2210_01837_gb300.workloads import rollers_1m  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "products/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_algorithmic_bytes_scale_with_fields_and_planes():
    params, pos, _, _ = rollers_1m(n=1 << 10, nxy=96, L=64.0)
    n = len(pos)
    a6 = bench.algorithmic(params, n, 20, 4, 400, fields=6)
    a3 = bench.algorithmic(params, n, 20, 4, 400, fields=3)
    a6z = bench.algorithmic(params, n, 40, 4, 400, fields=6)
    nx, ny = params["nx"], params["ny"]
    real6 = 6 * 20 * ny * nx * 4
    cpx6 = 6 * 20 * ny * (nx // 2 + 1) * 2 * 4
    # the xy FFT passes move only grid values: proportional to fields and to occupied planes
    for k in ("fft_x_fwd", "fft_y_fwd", "fft_y_inv", "fft_x_inv"):
        assert a6[k] == 2 * a3[k]
        assert a6z[k] == 2 * a6[k]
    assert a6["fft_x_fwd"] == real6 + cpx6 and a6["fft_y_fwd"] == 2 * cpx6
    # the spread writes the real grid once and reads every record once
    assert a6["spread"] - a3["spread"] == real6 // 2
    # the FP64 solve does not depend on the fields transformed
    assert a6["solve_fp64_flops"] == a3["solve_fp64_flops"] > 0
