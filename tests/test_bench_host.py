"""Host-side logic of bench.py (no GPU): the reference arm's JSON line and
the rule that attaches committed ncu traffic to a bench line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_json_line():
    # the reference arm times the CPU oracle: one benchmark step after the
    # minimum of three warm-up steps (about 20 s on 8 cores)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["higher_is_better"] is True and line["vs_baseline"] is None and line["dtype"] == "f64"
    assert "1024x512x512" in line["config"]["workload"]
    assert "1024x512x8" in line["cpu_baseline"]["sample"] and line["config"]["sample_nodes"] == 1024 * 512 * 8
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    e = line["e2e"]
    assert e["value"] == line["value"] and e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_traffic_record_matching(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"workloads": {
        "grid256/f32/ab": {"kernel_source_sha256": "K", "dram_bytes_per_launch_full_size": 1.0},
        "grid256/f32/ab/fused": {"kernel_source_sha256": "F", "fused_fz": 19, "fused_group": 1,
                                 "dram_bytes_per_launch_full_size": 2.0},
        "grid1024/f32/ab/fused": [
            {"kernel_source_sha256": "F", "fused_fz": 12, "fused_group": 4, "dram_bytes_per_launch_full_size": 3.0},
            {"kernel_source_sha256": "old", "fused_fz": 16, "fused_group": 2, "dram_bytes_per_launch_full_size": 4.0}]}}
    (prof / "collide_stream_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_digest", lambda fused=False: "F" if fused else "K")
    assert bench.ncu_traffic("grid256", "f32", "ab") == 1.0
    assert bench.ncu_traffic("grid256", "f32", "ab", True, 19, 1) == 2.0
    assert bench.ncu_traffic("grid256", "f32", "ab", True, 16, 1) is None       # other launch shape
    assert bench.ncu_traffic("grid1024", "f32", "ab", True, 12, 4) == 3.0
    assert bench.ncu_traffic("grid1024", "f32", "ab", True, 16, 2) is None      # taken on other sources
    assert bench.ncu_traffic("grid256", "f32", "aa") is None                    # no record
    monkeypatch.setattr(bench, "kernel_digest", lambda fused=False: "changed")
    assert bench.ncu_traffic("grid256", "f32", "ab") is None                    # kernel changed since


def test_committed_traffic_records_are_well_formed():
    with open(os.path.join(ROOT, "profiles", "collide_stream_traffic.json")) as fh:
        d = json.load(fh)
    assert "grid256/f32/ab/fused" in d["workloads"]
    for key, e in d["workloads"].items():
        for r in (e if isinstance(e, list) else [e]):
            assert r["dram_bytes_per_launch_full_size"] > 0 and r["kernel_source_sha256"], key
            if key.endswith("/fused"):
                assert r["fused_fz"] > 0 and r["fused_group"] > 0, key
            # records of the current kernels: measured traffic within 20 % of
            # the algorithmic bytes (no large re-reads; kept records of
            # earlier sources or launch shapes may show more)
            if r["kernel_source_sha256"] == bench.kernel_digest(key.endswith("/fused")):
                ratio = r["dram_bytes_per_launch_full_size"] / r["algorithmic_bytes_per_launch"]
                assert 0.8 <= ratio <= 1.2, (key, ratio)


def test_kernel_digest_follows_the_code_not_the_comments():
    import bench
    base = {"lbm_node.cuh": "int a; // one\n", "lbm_fused_kernel.cuh": "/* two\n lines */ int b;\n",
            "lbm_device.cuh": "int c;\n\n"}
    d0 = bench.kernel_digest(True, read=base.get)
    commented = dict(base, **{"lbm_node.cuh": "// a new comment\nint a;   // other words\n\n"})
    assert bench.kernel_digest(True, read=commented.get) == d0
    changed = dict(base, **{"lbm_device.cuh": "int c = 1;\n"})
    assert bench.kernel_digest(True, read=changed.get) != d0
