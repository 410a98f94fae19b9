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


def test_field_error_is_relative_to_the_field_itself():
    b = np.array([1e-6, -2e-6])
    a = b + 1e-9
    assert abs(bench.field_err(a, b) - 1e-9 / 2e-6) < 1e-15
    other = np.array([1.0, 0.5])
    assert abs(bench.field_err(other + 1e-6, other) - 1e-6) < 1e-15


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
    counts, src = bench.oracle_counts("n63")
    assert counts["evaluations"] >= 2 and counts["gmres_its"] > 0 and "oracle" in src
    t_par = bench.cpu_solve_estimate(s, counts, 16)
    t_one = bench.cpu_solve_estimate(s["single"], counts, 16)
    assert 0 < t_par < t_one
    assert bench.host_cores() >= 1


def test_timed_oracle_solve_equals_the_serial_oracle():
    """bench.py's timed CPU baseline is the oracle's own solve, spread over
    processes: same counts as the serial oracle, and a positive CPU time."""
    from oracle import discretization as fd, ras as oras, solvers
    from paper_2411_00546_gb300 import inputs
    o = bench.oracle_solve_timed("n63", 2)
    cfg = inputs.problem("n63")
    prob = fd.Problem(cfg["n"], cfg["phi"], cfg["nu"], cfg["mu"], inputs.make_yd(cfg))
    ref = solvers.raspen(prob, cfg["sx"], cfg["sy"], cfg["overlap"],
                         oras.Options(tol=cfg["tol"], inner_tol=cfg["inner_tol"], sigma=cfg["sigma"],
                                      eps0=cfg["eps0"], gamma=cfg["gamma"], eps_min=cfg["eps_min"]))
    np.testing.assert_array_equal(o["Y"], ref.Y)
    np.testing.assert_array_equal(o["P"], ref.P)
    assert o["outer"] == ref.outer and o["gmres_its"] == ref.gmres_its
    assert o["inner_its_per_eval"] == [sum(i) for i in ref.inner_its]
    assert o["workers"] == 2 and o["wall_s"] > 0 and o["cpu_s"] > 0


def test_bench_names_are_all_defined():
    """Every global name bench.py reads is defined in it or imported (its GPU
    legs run only on a GPU, so a missing constant would surface only there)."""
    import ast
    import builtins
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    defined = set(dir(builtins)) | {"__file__"}
    for node in ast.walk(tree):
        if isinstance(node, (ast.FunctionDef, ast.ClassDef)):
            defined.add(node.name)
        elif isinstance(node, (ast.Import, ast.ImportFrom)):
            defined.update((a.asname or a.name).split(".")[0] for a in node.names)
        elif isinstance(node, ast.arg):
            defined.add(node.arg)
        elif isinstance(node, ast.ExceptHandler) and node.name:
            defined.add(node.name)
        elif isinstance(node, ast.Name) and isinstance(node.ctx, ast.Store):
            defined.add(node.id)
    used = {n.id for n in ast.walk(tree) if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load)}
    assert sorted(used - defined) == []


def test_default_run_leaves_the_long_studies_to_flags(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse_args()
    assert (a.gpus, a.full, a.paper_methods, a.paper_layouts) == (1, False, False, None)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--full", "--paper-methods", "--paper-layouts", "2x2,2x5"])
    a = bench.parse_args()
    assert a.full and a.paper_methods and a.paper_layouts.split(",") == ["2x2", "2x5"]
