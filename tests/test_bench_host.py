"""Host logic of the measurement script: which clock records disqualify a
timed region (it is then measured once more)."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_clock_record_rejection():
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    assert bench.clocks_rejected(ok) == ""
    assert bench.clocks_rejected({**ok, "reasons": ["sw_power_cap"]}) == ""    # kept and noted
    assert bench.clocks_rejected({**ok, "reasons": ["hw_slowdown"]}) == "hw_slowdown"
    assert bench.clocks_rejected({**ok, "reasons": ["sw_power_cap", "sw_thermal_slowdown",
                                                    "hw_thermal_slowdown"]}) == "hw_thermal_slowdown,sw_thermal_slowdown"
    assert "no reason" in bench.clocks_rejected({**ok, "sm_mhz": 1200.0})     # a leftover clock lock
    assert bench.clocks_rejected({**ok, "sm_mhz": 1200.0, "reasons": ["sw_power_cap"]}) == ""
    assert bench.clocks_rejected({"sm_mhz": None, "sm_max_mhz": None, "reasons": []}) == ""   # no samples
