"""Host-side pieces of bench.py, on the CPU: the reference arm's JSON line
(it times the oracle, so it needs no GPU), the gate that drops a committed
DRAM-traffic figure once the kernel sources change, and the sort byte model."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "uniform3d_200", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "nnz/s" and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["metric"] == bench.METRIC and d["dtype"] == "f64"
    assert d["config"]["workload"].startswith("uniform3d_200")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "uniform3d_200", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_traffic_figure_needs_matching_sources(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "mttkrp_toy_traffic.txt").write_text(
        "# header\nkernel: k_stream\nkernel_source_sha256_16: abcdef0123456789\n"
        "dram_bytes_per_launch_mean: 3.5e+09\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda kernel: "abcdef0123456789")
    assert bench.profiled_traffic("mttkrp", "toy") == pytest.approx(3.5e9)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda kernel: "0000000000000000")
    assert bench.profiled_traffic("mttkrp", "toy") is None  # sources changed since the capture
    assert bench.profiled_traffic("mttkrp", "absent") is None


def test_committed_traffic_files_name_their_kernel_sources():
    for k in bench.KERNEL_SOURCES:
        p = os.path.join(ROOT, "profiles", f"{k}_zipf3d_traffic.txt")
        kv = dict(l.split(":", 1) for l in open(p) if ":" in l and not l.startswith("#"))
        assert len(kv["kernel_source_sha256_16"].strip()) == 16
        assert float(kv["dram_bytes_per_launch_mean"]) > 1e9


def test_sort_byte_model():
    r = bench.sort_roofline([2.0, 1.0, 1.0], nnz=1_000_000, N=3, peak=1000.0)
    alg = 1_000_000 * (8 * 3 + 8)  # read and write N indices + value, 4 bytes each
    assert r["alg_bytes_per_mode"] == alg
    assert r["achieved_gbs"] == pytest.approx(alg / (4 / 3 * 1e-3) / 1e9, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved_gbs"] / 1000.0, rel=1e-3)


def test_mttkrp_byte_model():
    # order 3, R = 32, FP32 factors: COO stream 16 B per entry, the other modes'
    # touched rows once, the FP32 output once
    touched = [900, 500, 300]
    dims = [1000, 600, 400]
    b = bench.mttkrp_alg_bytes(10_000, 3, 32, 4, touched, dims, 1)
    assert b == 10_000 * 16 + (900 + 300) * 32 * 4 + 600 * 32 * 4
    # 16-bit factors halve the row bytes, not the stream or the FP32 output
    b16 = bench.mttkrp_alg_bytes(10_000, 3, 32, 2, touched, dims, 1)
    assert b16 == 10_000 * 16 + (900 + 300) * 32 * 2 + 600 * 32 * 4


def test_sharded_ranges_cover_every_copy_position():
    from paper_1902_03317_gb300 import shard
    for nnz in (0, 5, 100_003):
        for world in (1, 2, 3, 8):
            got = [shard.step_range(nnz, world, r) for r in range(world)]
            assert got == shard.aligned_ranges(nnz, world)
            covered = sum(hi - lo for lo, hi in got)
            assert covered == nnz and all(lo % 4 == 0 for lo, _ in got)
