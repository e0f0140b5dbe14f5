"""Host logic of bench.py that needs no GPU: the DRAM-traffic record of the
packed GEMM is reported only while the kernel sources hash to the recorded
value and the timed plan uses the recorded W."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _record(tmp_path, sha, W=2, traffic=123456):
    p = tmp_path / "traffic.md"
    p.write_text(f"# summary\n\nsome text\n\nW: {W}\ntraffic_bytes_per_launch: {traffic}\n"
                 f"sources_sha256: {sha}\n")
    return str(p)


def test_traffic_reported_while_sources_match(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_FILE", _record(tmp_path, bench.gemm_sources_sha256()))
    assert bench.gemm_traffic(2) == 123456.0


def test_traffic_null_after_a_source_change(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_FILE", _record(tmp_path, "0" * 64))
    assert bench.gemm_traffic(2) is None


def test_traffic_null_for_another_packing(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_FILE", _record(tmp_path, bench.gemm_sources_sha256()))
    assert bench.gemm_traffic(3) is None


def test_traffic_null_without_a_record(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.md"))
    assert bench.gemm_traffic(2) is None


def test_source_hash_covers_every_listed_file():
    h1 = bench.gemm_sources_sha256()
    assert len(h1) == 64 and h1 == bench.gemm_sources_sha256()
    csrc = os.path.join(ROOT, "paper_1110_5765_gb300", "csrc")
    for name in bench.GEMM_SOURCES:
        assert os.path.exists(os.path.join(csrc, name)), name
