"""Host-side helpers of bench.py on CPU: the error metric of the mixed-vs-FP64
comparison, the captured-traffic lookup keyed by source hashes (whole files
and header regions), and the reference arm's JSON line."""
import hashlib
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_field_error_floors_a_small_field_at_the_joint_scale():
    b = np.array([1e-6, -2e-6])
    other = np.array([1.0, 0.5])
    a = b + 1e-9
    # scale max(2e-6, 1e-2 * 1.0) = 1e-2
    assert abs(bench.field_err(a, b, other) - 1e-9 / 1e-2) < 1e-18
    # a field on its own scale
    assert abs(bench.field_err(other + 1e-6, other, b) - 1e-6) < 1e-15


def test_traffic_lookup_follows_the_hashed_sources(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    hdr = tmp_path / "k.cuh"
    src.write_text("kernel body\n")
    hdr.write_text("// head\nstruct A { int x; };\n// tail marker\nother declarations\n")
    region = "struct A { int x; };\n"
    table = {"jvp": {"bytes_per_launch": 123.0, "workload": "w",
                     "sources": [("k.cu", None, None), ("k.cuh", "struct A {", "// tail marker")],
                     "sha256": [hashlib.sha256(b"kernel body\n").hexdigest(),
                                hashlib.sha256(region.encode()).hexdigest()]}}
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC", table)
    assert bench.traffic_for("jvp", "w") == 123.0
    assert bench.traffic_for("jvp", "other workload") is None
    assert bench.traffic_for("factor", "w") is None
    # a change outside the hashed header region keeps the figure
    hdr.write_text("// head\nstruct A { int x; };\n// tail marker\nmore declarations\n")
    assert bench.traffic_for("jvp", "w") == 123.0
    # a change inside it, or in the kernel's file, drops it
    hdr.write_text("// head\nstruct A { long x; };\n// tail marker\n")
    assert bench.traffic_for("jvp", "w") is None
    hdr.write_text("// head\nstruct A { int x; };\n// tail marker\n")
    src.write_text("kernel body changed\n")
    assert bench.traffic_for("jvp", "w") is None


def test_whole_job_rate():
    assert bench.whole_job_rate(4, 3, 1.5) == pytest.approx(8.0)


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600, check=True).stdout
    line = json.loads(out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["value"] > 0 and line["unit"] == "solves/s" and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_parallel_cpu_sample_scales_the_throughput():
    s = bench.run_cpu_sample_parallel("n63", 2)
    assert s["cores"] == 2 and s["subdomains"] == 2
    assert s["inner_its"] == 2 * s["single"]["inner_its"]
    assert s["solve_s"] == pytest.approx(s["single"]["solve_s"] / 2, rel=1.0)
    counts = {"inner_its_sum": 100, "evaluations": 2, "gmres_its": 10}
    t_par = bench.cpu_solve_estimate(s, counts, 16)
    t_one = bench.cpu_solve_estimate(s["single"], counts, 16)
    assert 0 < t_par < t_one
    assert bench.host_cores() >= 1
