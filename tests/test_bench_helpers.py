"""Host-side helpers of bench.py (no GPU): the pair-scaled DRAM traffic of the
roofline line and the job throughput."""
import hashlib
import json
import os

import bench


def _fake_tree(tmp_path, src_text=b"kernel source"):
    csrc = tmp_path / "paper_2604_10982_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_bytes(src_text)
    (tmp_path / "profiles").mkdir()
    h = hashlib.sha256(src_text).hexdigest()[:16]
    entry = {"sources": ["k.cu"], "sha256_16": h, "view": "1920x1080",
             "points": [{"pairs": 1000, "dram_read": 150_000, "dram_write": 50_000},
                        {"pairs": 3000, "dram_read": 350_000, "dram_write": 50_000}]}
    (tmp_path / "profiles" / "roofline_traffic.json").write_text(json.dumps({"k_kernel": entry}))
    return csrc


def test_traffic_is_the_line_through_the_two_captures(tmp_path, monkeypatch):
    _fake_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # 200 kB at 1000 pairs, 400 kB at 3000: 100 B per pair + 100 kB
    b, note = bench.roofline_traffic("k_kernel", 2000.0, "1920x1080")
    assert abs(b - 300_000.0) < 1e-6, note
    b, _ = bench.roofline_traffic("k_kernel", 0.0, "1920x1080")
    assert abs(b - 100_000.0) < 1e-6


def test_traffic_refused_when_sources_or_view_differ(tmp_path, monkeypatch):
    csrc = _fake_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    b, why = bench.roofline_traffic("k_kernel", 2000.0, "1280x720")
    assert b is None and "1920x1080" in why
    b, why = bench.roofline_traffic("other_kernel", 2000.0, "1920x1080")
    assert b is None and "other_kernel" in why
    (csrc / "k.cu").write_bytes(b"kernel source, edited")
    b, why = bench.roofline_traffic("k_kernel", 2000.0, "1920x1080")
    assert b is None and "changed" in why


def test_job_throughput_counts_every_rank():
    # 2 ranks x 10 steps in 500 ms (the slowest rank) = 40 units/s
    assert abs(bench.job_throughput(10, 2, 500.0) - 40.0) < 1e-12
