"""Host-side helpers of bench.py that shape its JSON line (no GPU): the
class roofline (achieved = algorithmic bytes over device time, fractions of
the measured and of the nominal peak, DRAM traffic per launch from the ncu
table), the hierarchy report, the solves/s arithmetic and the peak lookup."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_class_roofline_picks_the_class_with_most_time():
    prof = {"setup_spgemm": (800.0, 8.0e10, 50), "hybrid_gs_sweep": (300.0, 1.0e12, 1000),
            "idle": (0.0, 0.0, 0)}
    r = bench.class_roofline(prof, 8000.0, "measured")
    assert r["kernel"] == "setup_spgemm"
    assert r["achieved"] == pytest.approx(8.0e10 / 0.8 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 8000.0)
    assert r["frac_nominal"] == pytest.approx(r["achieved"] / bench.NOMINAL_HBM_GBS)
    assert r["launch_ms"] == pytest.approx(16.0) and r["bytes_per_launch"] == pytest.approx(1.6e9)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak_source"] == "measured"
    # the ncu traffic of a class is reported per launch
    if "setup_spgemm" in bench.NCU_TRAFFIC:
        assert r["traffic"] == pytest.approx(bench.NCU_TRAFFIC["setup_spgemm"][0] / 50)
    # restricted to the solve classes
    s = bench.class_roofline(prof, 8000.0, "measured", classes=("hybrid_gs_sweep",))
    assert s["kernel"] == "hybrid_gs_sweep" and s["frac"] == pytest.approx(1.0e12 / 0.3 / 1e9 / 8000.0)
    assert s["traffic"] is None or "hybrid_gs_sweep" in bench.NCU_TRAFFIC
    assert bench.class_roofline({"idle": (0.0, 0.0, 0)}, 8000.0, "measured") is None
    json.dumps(r)


def test_hierarchy_stats_operator_complexity():
    class H:
        nlevels = 3

        def level_info(self, l):
            return [(1000, 5000, 3000, 6), (300, 2400, 600, 9), (40, 600, 0, 0)][l]

    class M:
        def amg(self, which):
            return H() if which == 0 else None

    out = bench.hierarchy_stats(M())
    assert list(out) == ["hierarchy_0"]
    assert out["hierarchy_0"]["levels"] == 3
    assert out["hierarchy_0"]["rows"] == [1000, 300, 40]
    assert out["hierarchy_0"]["op_complexity"] == pytest.approx((5000 + 2400 + 600) / 5000)


def test_solves_per_second_and_peak():
    assert bench.solves_per_second(2, 5, 10000.0) == pytest.approx(1.0)
    assert bench.solves_per_second(2, 5, 0.0) == 0.0
    peak, kind = bench.hbm_peak()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and peak == pytest.approx(float(json.load(open(path))["hbm_gbs"]))
    else:
        assert kind == "fallback" and peak == 6800.0
