"""The benchmark's clock check (host logic, no GPU): which clock records
disqualify a timed region's number and send it to be measured once more."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_throttle_reasons_reject():
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_rejected({"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [r]})


def test_power_cap_alone_is_kept():
    assert not bench.clocks_rejected({"sm_mhz": 1650.0, "sm_max_mhz": 2070.0,
                                      "reasons": ["sw_power_cap"]})


def test_low_clock_without_a_reason_rejects():
    # a clock lock left by someone else: well below max, nothing active
    assert bench.clocks_rejected({"sm_mhz": 1400.0, "sm_max_mhz": 2070.0, "reasons": []})
    assert not bench.clocks_rejected({"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []})
    assert not bench.clocks_rejected({"sm_mhz": 1950.0, "sm_max_mhz": 2070.0, "reasons": []})


def test_no_samples_is_not_a_rejection():
    assert not bench.clocks_rejected({"sm_mhz": None, "sm_max_mhz": None,
                                      "reasons": ["no samples"]})
