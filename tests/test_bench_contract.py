"""The JSON line of bench.py's reference arm (the oracle timed on the host)
and the helpers the GPU arm uses to report DRAM traffic, checked on CPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--config", "1", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["m"] == 32768


def test_traffic_table_lookup(tmp_path, monkeypatch):
    sha = bench.kernel_source_sha()
    assert len(sha) == 16 and sha == bench.kernel_source_sha()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "ncu_traffic.txt").write_text(
        "# comment\n"
        f"k_solve {sha} 123 grid2d_1024x1024\n"
        f"k_solve 0000000000000000 999 rmat_scale22\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: sha)
    assert bench.traffic_for("k_solve", "grid2d_1024x1024") == 123.0
    assert bench.traffic_for("k_solve", "rmat_scale22") is None   # other kernel source
    assert bench.traffic_for("k_solve", None) is None
    assert bench.traffic_for("k_other", "grid2d_1024x1024") is None


def test_batched_traffic_scales_by_edges(tmp_path, monkeypatch):
    sha_b = bench.kernel_source_sha(files=bench.BATCHED_FILES)
    assert len(sha_b) == 16 and sha_b != bench.kernel_source_sha()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "ncu_traffic.txt").write_text(
        f"k_solve {sha_b} 5 grid2d_1024x1024\n"
        f"k_b_solve 0000000000000000 7 edges=10 other_code\n"
        f"k_b_solve {sha_b} 1000 edges=250 batched_small\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_sha", lambda files=None: sha_b)
    traffic, src = bench.batched_traffic_for(1000)
    assert traffic == 4000.0 and "250-edge batch" in src  # 1000 B for 250 edges, x4
    assert bench.batched_traffic_for(0) == (None, None)
    monkeypatch.setattr(bench, "kernel_source_sha", lambda files=None: "f" * 16)
    assert bench.batched_traffic_for(1000) == (None, None)  # captured on other code


@pytest.mark.parametrize("xs,p50,p99", [([], None, None), ([5.0], 5.0, 5.0),
                                        (list(range(1, 101)), 51, 99)])
def test_percentiles(xs, p50, p99):
    assert bench._percentiles(xs) == (p50, p99)


def test_cpu_baselines_on_a_small_graph():
    from paper_2005_06913_gb300 import graphgen as gg
    g = gg.random_connected(2000, 8000, 3)
    seq = bench.cpu_baseline(g, budget_s=0.05)
    par = bench.cpu_parallel_baseline(g, budget_s=0.05)
    assert seq["kind"] == "oracle" and seq["cores"] == 1 and seq["value"] > 0
    assert par["cores"] >= 1 and par["value"] > 0 and "2.2.2" in par["kind"]
    assert par["unit"] == seq["unit"] == bench.UNIT
    assert seq["host"]["arch"] and seq["host"]["cores_available"] >= 1

