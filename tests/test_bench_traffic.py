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


def test_recorded_traffic_matches_the_current_sources():
    """Both committed captures were taken on the current kernel code, so the
    bench reports their traffic: bytes per event times the events."""
    for wl in ("256x256_bt4", "2048x2048_bt16"):
        t = bench.tile_traffic(wl, 1.0e6)
        assert t is not None, wl
        assert 15.0e6 < t < 21.0e6, (wl, t)  # 15-21 DRAM bytes per event, one read and one write a key


def test_stale_capture_reports_no_traffic(monkeypatch):
    monkeypatch.setattr(bench, "tile_source_hash", lambda: "0" * 64)
    assert bench.tile_traffic("256x256_bt4", 1.0e6) is None
    assert bench.tile_traffic("no_such_workload", 1.0e6) is None
