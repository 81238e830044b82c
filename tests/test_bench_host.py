"""Host logic of bench.py that decides what a JSON line may claim, checked
without a GPU: the clock record (a run with a thermal or hardware slowdown
is rejected, a power cap is kept and noted) and the DRAM traffic figure taken
from the committed ncu summary only while that summary matches the kernel
source it was captured from."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(lines):
    c = bench.ClockSampler(0)
    c.proc = _FakeProc()
    c.lines = list(lines)
    return c


def _line(sm, smax, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return "0, %d, %d, 812.40, 0x0000000000000000, %s, %s, %s, %s" % (sm, smax, hw, hwt, swt, cap)


def test_clock_record_median_max_and_no_reason():
    rec = _sampler([_line(2070, 2070), _line(2055, 2070), _line(2070, 2070)]).stop()
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == [] and rec["samples"] == 3


def test_clock_record_names_every_active_reason():
    rec = _sampler([_line(1980, 2070, cap="Active"), _line(1500, 2070, hwt="Active"),
                    _line(2070, 2070, hw="Active", swt="Active")]).stop()
    assert rec["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert rec["sm_mhz"] == 1980.0


def test_clock_record_skips_malformed_lines_and_reports_a_missing_tool():
    rec = _sampler(["", "garbage", "0, [N/A], 2070, 1, 0x0, Not Active, Not Active, Not Active, Not Active",
                    _line(2070, 2070)]).stop()
    assert rec["samples"] == 1 and rec["sm_mhz"] == 2070.0
    none = bench.ClockSampler(0).stop()       # never started: no nvidia-smi process
    assert none["sm_mhz"] is None and none["reasons"] == ["nvidia-smi unavailable"]


def _profile_fields():
    fields = {}
    with open(bench.SWEEP_PROFILE) as f:
        for line in f:
            if ":" in line:
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
    return fields


def test_traffic_comes_from_the_summary_only_while_it_matches_the_source():
    f = _profile_fields()
    kernel, workload = f["kernel"], f["workload"]
    got = bench.sweep_traffic(kernel.split("::")[-1], workload)
    if f["source_digest"] == bench.source_digest(bench.SWEEP_SOURCE):
        assert got == float(f["traffic_bytes_per_launch"])
    else:
        assert got is None                    # the kernel changed since the capture
    assert bench.sweep_traffic(kernel.split("::")[-1], "another_workload") is None
    assert bench.sweep_traffic("k_some_other_kernel", workload) is None

