"""The benchmark's JSON line on the GPU, on small cases of each workload: one
line with every key of the line contract (roofline with its measured peak,
cpu_baseline, e2e with its host<->device bytes, clocks, gpu_launches)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def run_bench(*extra):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "12", "--warmup", "3"] + list(extra)
    r = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-3000:]
    return json.loads(lines[0])


def check_contract(d, bound):
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
                "gpu_launches", "clocks"):
        assert key in d, key
    assert d["n_gpus"] == 1 and d["steps"] == 12 and d["warmup"] == 3
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["gpu_launches"] >= d["steps"]
    assert d["config"]["workload"]
    r = d["roofline"]
    assert r["bound"] == bound and r["achieved"] > 0 and r["peak"] > 0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    assert "traffic" in r and r["unit"] in ("GB/s", "TFLOP/s")
    c = d["cpu_baseline"]
    assert c["kind"] == "oracle" and c["value"] > 0 and c["cores"] >= 1 and c["sample"]
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert "sm_mhz" in d["clocks"] and "reasons" in d["clocks"]


def test_default_workload_line():
    d = run_bench("--nz", "128", "--e2e-steps", "40")
    check_contract(d, "hbm")
    assert d["dtype"] == "f32" and d["roofline"]["kernel"].startswith("fused_step")


def test_rz_workload_line():
    d = run_bench("--workload", "rz", "--nz", "1024", "--e2e-steps", "40")
    check_contract(d, "hbm")


def test_yee_line_carries_the_scheme_comparison():
    d = run_bench("--scheme", "yee", "--nz", "128", "--e2e-steps", "40")
    check_contract(d, "hbm")
    v = d["versus_tetm"]
    assert v["tetm_kernel_ms_per_step"] > 0 and v["yee_ms_per_dz"] > 0
    z = d["z_dispersion"]
    assert z["tetm"]["max_error_vs_dispersion_free"] < 1e-10
    assert z["yee"]["max_error_vs_eq10"] < 1e-10 < z["yee"]["max_error_vs_dispersion_free"]
