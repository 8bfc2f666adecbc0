"""Host-side arithmetic of bench.py (no GPU): the job's throughput over
ranks and the HBM fraction of a throughput."""
import json
import os

import pytest

import bench


def test_hbm_fraction_uses_the_measured_peak():
    peak, kind = bench._peaks()
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and peak == pytest.approx(float(json.load(open(path))["hbm_gbs"]))
    else:
        assert kind == "fallback"
    # 1000 MP/s/iter at 56 B/px/iter moves 56 GB/s
    assert bench._hbm_frac(1000.0, 56.0) == pytest.approx(56.0 / peak)


def test_job_value_counts_all_ranks_work():
    # 4 ranks x 2.0 MP-iterations per step x 10 steps in 20 ms
    assert bench._job_value(4, 2.0, 10, 20.0) == pytest.approx(4 * 2.0 * 10 / 0.020)
