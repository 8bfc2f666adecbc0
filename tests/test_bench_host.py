"""Host-side arithmetic of bench.py (no GPU): the job's throughput over
ranks, the HBM fraction of a throughput, the counted work model of a pass
and the validity check of the recorded DRAM traffic."""
import json
import os

import pytest

import bench


def test_hbm_fraction_uses_the_measured_peak():
    peak, sm_mhz, kind = bench._peaks()
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        assert kind == "measured" and peak == pytest.approx(float(d["hbm_gbs"]))
        assert sm_mhz == pytest.approx(float(d.get("sm_max_mhz", bench.FALLBACK_SM_MHZ)))
    else:
        assert kind == "fallback"
    # 1000 MP/s/iter at 56 B/px/iter moves 56 GB/s
    assert bench._hbm_frac(1000.0, 56.0) == pytest.approx(56.0 / peak)


def test_job_value_counts_all_ranks_work():
    # 4 ranks x 2.0 MP-iterations per step x 10 steps in 20 ms
    assert bench._job_value(4, 2.0, 10, 20.0) == pytest.approx(4 * 2.0 * 10 / 0.020)


def test_pass_bytes():
    # RGB FP32 with an FP32 guidance: 12 B in, 12 B out, 4 B guidance per pixel
    assert bench.pass_bytes(1080, 1920, 3) == 1080 * 1920 * 28
    assert bench.pass_bytes(1080, 1920, 3, 2, 2) == 1080 * 1920 * 14


def test_flops_per_entry_term_by_term():
    # r = 1, C = 3: weights 4, diagonal 2, LDL^T row 0 + 1 + 2, substitutions
    # 6 + (6 + 3), accumulation 3
    assert bench.flops_per_entry(1, 3) == 4 + 2 + 3 + 6 + 9 + 3
    # r = 2, C = 3: 8 + 4 + (2 + 2 + 4) + 12 + 15 + 3
    assert bench.flops_per_entry(2, 3) == 50
    assert bench.mufu_per_entry(2) == 3


def test_pass_work_counts_every_entry():
    # column pass of 1920 x 1080 at r = 2: 1916 centres x 5 x 1080 entries
    fl, mu = bench.pass_work(1080, 1920, 3, 2, 0)
    assert fl == 1916 * 5 * 1080 * 50 and mu == 1916 * 5 * 1080 * 3
    fl, mu = bench.pass_work(1080, 1920, 3, 2, 1)
    assert fl == 1076 * 5 * 1920 * 50


def test_alu_peaks():
    f, m = bench.alu_peaks(2070.0)
    assert f == pytest.approx(152 * 128 * 2 * 2.07e9)
    assert m == pytest.approx(152 * 16 * 2.07e9)


def test_traffic_only_for_the_current_sources(tmp_path, monkeypatch):
    path = tmp_path / "traffic.txt"
    path.write_text(f"# comment\nsource_hash {bench.source_hash()}\nwl row 123.0\nwl column 456\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(path))
    assert bench.measured_traffic("wl", "row") == 123.0
    assert bench.measured_traffic("wl", "column") == 456.0
    assert bench.measured_traffic("other", "row") is None
    path.write_text("source_hash 0000000000000000\nwl row 123.0\n")
    assert bench.measured_traffic("wl", "row") is None   # counters of other kernels
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.txt"))
    assert bench.measured_traffic("wl", "row") is None


def test_roofline_lines_pick_the_slower_direction():
    hbm, alu = bench.roofline_lines(1080, 1920, 3, 2, col_ms=0.1, row_ms=0.2, workload="none")
    assert hbm["kernel"].startswith("row") and alu["kernel"].startswith("row")
    peak, sm_mhz, _ = bench._peaks()
    assert hbm["achieved"] == pytest.approx(1080 * 1920 * 28 / 0.2e-3 / 1e9)
    assert hbm["frac"] == pytest.approx(hbm["achieved"] / peak)
    fl, _ = bench.pass_work(1080, 1920, 3, 2, 1)
    assert alu["achieved"] == pytest.approx(fl / 0.2e-3 / 1e12)
    assert alu["frac"] == pytest.approx(fl / 0.2e-3 / bench.alu_peaks(sm_mhz)[0])


def test_source_hash_ignores_comments_only():
    """The traffic file stays valid across comment edits, not code edits."""
    code = "int a = 1;  // one\n/* block\n comment */\nint b = 2;\n"
    assert bench.code_only(code) == bench.code_only("int a = 1;\n\n// other words\nint b = 2;")
    assert bench.code_only(code) != bench.code_only("int a = 1;\nint b = 3;")
