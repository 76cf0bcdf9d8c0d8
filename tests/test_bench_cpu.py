"""The benchmark's reference arm (the oracle on a bounded sample of each
workload) runs on the host: one JSON line with the keys the line contract
names, for the Cartesian, rotationally symmetric and Yee workloads."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_reference(*extra):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
           "--warmup", "1", "--nz", "48"] + list(extra)
    r = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


@pytest.mark.parametrize("extra", [(), ("--scheme", "yee"), ("--workload", "rz")])
def test_reference_arm_line(extra):
    d = run_reference(*extra)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "gpu_launches"):
        assert key in d, key
    assert d["impl"] == "reference" and d["gpu_launches"] == 0
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"]


def test_profiled_traffic_needs_the_profiled_source_and_work_shape(tmp_path, monkeypatch):
    """The line's `traffic` comes from a committed ncu summary only while the
    kernel source hashes as it did when the summary was taken, and (when the
    summary names one) only for the work shape it was taken at."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = tmp_path / "paper_0901_1053_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "k.cu").write_text("// a kernel\n")
    h = bench.kernel_source_hash(("k.cu",))
    assert len(h) == 16 and h == bench.kernel_source_hash(("k.cu",))
    (tmp_path / "profiles" / "p.md").write_text(
        "# k\n\nkernel_source_sha256_16: %s\ntiling: 56, 28, 45\ntraffic_bytes_per_launch: 1.5e9\n" % h)
    assert bench.profiled_traffic("p.md", ("k.cu",), (56, 28, 45)) == 1.5e9
    assert bench.profiled_traffic("p.md", ("k.cu",)) == 1.5e9
    assert bench.profiled_traffic("p.md", ("k.cu",), (56, 28, 16)) is None   # another work shape
    assert bench.profiled_traffic("missing.md", ("k.cu",), (56, 28, 45)) is None
    (csrc / "k.cu").write_text("// the kernel, changed\n")
    assert bench.kernel_source_hash(("k.cu",)) != h
    assert bench.profiled_traffic("p.md", ("k.cu",), (56, 28, 45)) is None  # another source
    # a summary without a tiling line holds for any work shape of its source
    h2 = bench.kernel_source_hash(("k.cu",))
    (tmp_path / "profiles" / "q.md").write_text(
        "kernel_source_sha256_16: %s\ntraffic_bytes_per_launch: 2e9\n" % h2)
    assert bench.profiled_traffic("q.md", ("k.cu",), (32, 8, 64)) == 2e9
