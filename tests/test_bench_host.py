"""Host-side pieces of bench.py that need no GPU: reading the DRAM traffic of
the step kernel from a profile summary, which counts only when the summary
was taken on the current kernel source."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def write_summary(tmp_path, source_hash, traffic_line):
    p = tmp_path / "summary.md"
    p.write_text("# kernel\n\n- kernel_source_hash: %s\n- duration_ms: 0.2\n%s\n" % (source_hash, traffic_line))
    return str(p)


def test_traffic_read_when_hash_matches(tmp_path):
    p = write_summary(tmp_path, bench.kernel_hash() + " (sources without comments)",
                      "- dram_bytes_per_launch: 1.62e9 (24.1 B x 67.24 M cells, scaled)")
    assert bench.profiled_traffic(p) == 1.62e9


def test_hash_ignores_comments(tmp_path, monkeypatch):
    a = tmp_path / "a.cuh"
    a.write_text("int f(int x) {  // one\n  return x + 1; /* two */\n}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", ["a.cuh"])
    h1 = bench.kernel_hash()
    a.write_text("int f(int x) {\n  // changed comment\n  return x + 1;\n}\n")
    assert bench.kernel_hash() == h1
    a.write_text("int f(int x) { return x + 2; }\n")
    assert bench.kernel_hash() != h1


def test_traffic_dropped_for_another_source(tmp_path):
    p = write_summary(tmp_path, "0000000000000000", "- dram_bytes_per_launch: 1.62e9")
    assert bench.profiled_traffic(p) is None


def test_traffic_missing_or_malformed(tmp_path):
    assert bench.profiled_traffic(str(tmp_path / "absent.md")) is None
    p = write_summary(tmp_path, bench.kernel_hash(), "- dram_bytes_per_launch: n/a")
    assert bench.profiled_traffic(p) is None
