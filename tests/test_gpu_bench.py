"""The bench line on a small workload: the JSON contract, and accuracy keys that hold
the solve's known error (the 129^3 bump has an exact potential: 6th-order error
1.2e-12 at h = 2/128; the variants against FP64 within their stated budgets). A bench
that measured one buffer and reported the accuracy of another fails here."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.gpu
def test_bench_line_on_the_129cube_bump():
    r = subprocess.run([sys.executable, "bench.py", "--workload", "bump", "--headline-only", "--steps", "3",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["unit"] == "grid points/s" and d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["steps"] == 3 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["config"]["grid"] == [129, 129, 129] and d["config"]["order"] == 6
    assert d["value"] > 0 and d["e2e"]["value"] > 0 and d["gpu_launches"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 8 * 129 ** 3 == d["e2e"]["d2h_bytes_per_step"]
    # the phi* stage alone does less work than the solve
    assert d["phi_star_solve"]["value"] > d["value"]
    rf = d["roofline"]
    assert rf["bound"] == "alu" and 0 < rf["frac"] < 1.2 and rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"])
    assert set(d["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}
    # FP64: g against the direct trapezoid sum, phi against the exact potential
    assert d["precision"]["g_vs_direct_sum"] < 1e-13
    assert d["precision"]["max_rel_error_vs_exact_potential"] < 1e-10
    # the variants against the FP64 solve of the same run
    assert d["df32"]["max_rel_error_vs_fp64"] < 1e-11
    for key in ("mixed_precision", "mixed_tf32x3", "mixed_df32_boundary"):
        assert 0 < d[key]["max_rel_error_vs_fp64"] < 1e-4, key
