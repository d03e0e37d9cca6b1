"""The measured-traffic field of the bench line (host logic, no GPU): the
DRAM bytes per event of a committed ncu capture apply only while the sweep
kernel's code still hashes to the value recorded with the capture, and the
hash covers the code, not its comments."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def test_code_lines_drop_comments_and_blank_lines():
    src = "int a;  // one\n\n  // a whole comment line\nint b; // two\n   \nint c;\n"
    assert bench.code_lines(src) == "int a;\nint b;\nint c;"
    assert bench.code_lines(src) == bench.code_lines(src.replace("one", "another remark"))
    assert bench.code_lines(src) != bench.code_lines(src.replace("int b;", "int b = 1;"))


def _record(wl):
    with open(os.path.join(bench.ROOT, "profiles", "k_tile_%s.md" % wl)) as f:
        line = [l for l in f.read().splitlines() if l.startswith("traffic_record:")][-1]
    return dict(kv.partition("=")[::2] for kv in line.split(":", 1)[1].split())


def test_recorded_traffic_is_applied_for_its_sources(monkeypatch):
    """Each committed capture gives bytes per event times the events for the
    sources it was taken on (15-21 DRAM bytes per event: one read and one
    write of each 8-byte key, plus list tails)."""
    for wl in ("256x256_bt4", "2048x2048_bt16"):
        rec = _record(wl)
        assert 15.0 < float(rec["dram_bytes_per_event"]) < 21.0, (wl, rec)
        monkeypatch.setattr(bench, "tile_source_hash", lambda: rec["sources_sha256"])
        assert bench.tile_traffic(wl, 1.0e6) == float(rec["dram_bytes_per_event"]) * 1.0e6


def test_stale_capture_reports_no_traffic(monkeypatch):
    monkeypatch.setattr(bench, "tile_source_hash", lambda: "0" * 64)
    assert bench.tile_traffic("256x256_bt4", 1.0e6) is None
    assert bench.tile_traffic("no_such_workload", 1.0e6) is None
