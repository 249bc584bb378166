"""Host-side pieces of bench.py that need no GPU: the nvidia-smi clock sample
parser that reports the median SM clock under load and the throttle reasons
seen during the timed region."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def sampler_with(tmp_path, rows):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as fh:
        fh.write("\n".join(rows) + "\n")
    return s


def test_clock_summary_median_and_no_reasons(tmp_path):
    na = "Not Active"
    rows = [f"0, {mhz}, 2070, 900.5, 0x0, {na}, {na}, {na}, {na}" for mhz in (2070, 1980, 2055)]
    out = sampler_with(tmp_path, rows).summary()
    assert out["sm_mhz"] == 2055 and out["sm_max_mhz"] == 2070 and out["samples"] == 3
    assert out["reasons"] == []


def test_clock_summary_reports_active_throttle_reasons(tmp_path):
    na, ac = "Not Active", "Active"
    rows = [f"0, 2070, 2070, 1390.0, 0x4, {na}, {na}, {na}, {ac}",
            f"0, 1800, 2070, 1400.0, 0x8, {ac}, {na}, {na}, {na}",
            "garbage line",
            f"0, 1900, 2070, 1200.0, 0x0, {na}, {na}, {ac}, {na}"]
    out = sampler_with(tmp_path, rows).summary()
    assert out["samples"] == 3                       # the unparsable line is skipped
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def test_clock_summary_without_samples(tmp_path):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "missing.csv")
    out = s.summary()
    assert out["sm_mhz"] is None and out["samples"] == 0 and out["reasons"] == []
