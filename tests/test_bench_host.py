"""Host-side pieces of bench.py that need no GPU: the kernel-source hash that
keys recorded DRAM counters, and the lookup that drops counters once the
kernel's sources change."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _fake_tree(tmp_path):
    csrc = tmp_path / "paper_2201_07325_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("tcgemm.cu", "dfloat.cuh", "device_common.cuh", "fmmlu_internal.h", "solve.cu"):
        (csrc / f).write_text(f"// {f}\n")
    (tmp_path / "profiles").mkdir()
    return csrc


def test_recorded_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    csrc = _fake_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash("schur_tc")
    rec = {"ellipsoid50k": {"schur_tc": {"source_hash": h, "dram_bytes_per_launch": 123}}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("schur_tc", "ellipsoid50k") == 123
    assert bench.recorded_traffic("schur_tc", "torus200k") is None
    # a change outside the kernel's translation unit keeps the counters
    (csrc / "solve.cu").write_text("// changed\n")
    assert bench.kernel_source_hash("schur_tc") == h
    assert bench.recorded_traffic("schur_tc", "ellipsoid50k") == 123
    # a change inside it (a header it includes counts) drops them
    (csrc / "dfloat.cuh").write_text("// changed\n")
    h2 = bench.kernel_source_hash("schur_tc")
    assert h2 != h
    assert bench.recorded_traffic("schur_tc", "ellipsoid50k") is None
    (csrc / "tcgemm.cu").write_text("// changed\n")
    assert bench.kernel_source_hash("schur_tc") not in (h, h2)


def test_unlisted_kernels_hash_all_sources(tmp_path, monkeypatch):
    csrc = _fake_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash("sweep_fwd")
    assert h == bench.kernel_source_hash()
    (csrc / "solve.cu").write_text("// changed\n")
    assert bench.kernel_source_hash("sweep_fwd") != h
