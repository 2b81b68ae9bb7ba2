"""Host-side logic of bench.py that decides reported numbers, checked without a GPU:
  * the roofline denominator of the mixed integral kernel (SM clocks per term) from its unit
    counts: the SFU (2 MUFU per term at 16 per SM per clock) and the issue slots;
  * the nvidia-smi clock sampler's parsing: median SM clock under load, the maximum clock and
    the throttle reasons seen during the timed region."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_clocks_per_term_from_unit_counts():
    # without a split both models are SFU-bound: 2 MUFU / 16 per SM per clock
    for mode, R in ((0, 2), (2, 2), (0, 1), (2, 1)):
        c, f = bench.clocks_per_term(mode, R, 0)
        assert f == 0.0 and c == pytest.approx(2 / 16)
    # the issue-slot limits: phase FMUL, prescale FMUL, 2 MUFU, 4 or 6 FFMA (I_z is not summed),
    # one shared load per R energies: classical (4 + 4 + 1/2)/128 = 0.066, spin-1/2
    # (4 + 6 + 1/2)/128 = 0.082
    assert (4 + 4 + 0.5) / 128 < 2 / 16 and (4 + 6 + 0.5) / 128 < 2 / 16
    # a 1/4 split at R = 2 moves 4 of every 16 terms to the FMA pipe (18 extra slots each):
    # SFU 2 * 3/4 / 16 = 0.094, issue (8.5 + 18/4)/128 = 0.102, so issue binds
    c, f = bench.clocks_per_term(0, 2, 4)
    assert f == pytest.approx(0.25) and c == pytest.approx((4 + 4 + 0.5 + 18 * 0.25) / 128)
    # a 1/6 split at R = 2 moves 2 of every 16 (indices 5 and 11): SFU 2 * 7/8 / 16 = 0.109 binds
    c, f = bench.clocks_per_term(0, 2, 6)
    assert f == pytest.approx(0.125) and c == pytest.approx(2 * 0.875 / 16)
    # the benchmark's peak: 152 SMs x 2070 MHz / 0.125 clocks per term
    assert bench.SM_COUNT * bench.SM_MAX_MHZ * 1e6 / (2 / 16) == pytest.approx(2.517e12, rel=1e-3)


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampled(rows):
    c = bench.Clocks(0)
    fd, c.path = __import__("tempfile").mkstemp(suffix=".csv")
    os.close(fd)
    with open(c.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    c.proc = _Done()
    return c.stop()


def test_clock_sampler_parses_load_and_reasons():
    idle = "0, 345, 2070, 120.5, 0x0000000000000001, Not Active, Not Active, Not Active, Not Active"
    load = ["0, 2070, 2070, 1012.3, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1180.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2040, 2070, 1201.7, 0x0000000000000004, Not Active, Not Active, Not Active, Active"]
    got = _sampled([idle] + load + [idle, "garbage line", ""])
    # idle samples (below half the highest clock) are not "under load"
    assert got["sm_mhz"] == 2055.0 and got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == ["sw_power_cap"] and got["samples"] == 5
    assert got["power_w_max"] == pytest.approx(1201.7)


def test_clock_sampler_reports_throttling_and_absence():
    rows = ["0, 1500, 2070, 900.0, 0x0000000000000048, Not Active, Active, Not Active, Not Active"] * 3
    assert _sampled(rows)["reasons"] == ["hw_thermal_slowdown"]
    empty = _sampled(["not a sample"])
    assert empty["sm_mhz"] is None and empty["reasons"] == ["no samples"]
    c = bench.Clocks(0)
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]
