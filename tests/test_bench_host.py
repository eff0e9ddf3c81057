"""Host-side pieces of bench.py that need no GPU: the clock record taken
during the timed region (median SM clock, maximum clock, throttle reasons
seen) and the scanned-pair count of a search."""
import numpy as np

import bench


class _Done:
    def terminate(self):
        pass

    def wait(self):
        return 0


def _sampler_with(tmp_path, lines):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    s.proc = _Done()
    return s


def test_clock_record_median_max_and_reasons(tmp_path):
    rows = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1995, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 950.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 950.5, 0x0, Not Active, Not Active, Not Active, Not Active",   # skipped
        "garbage",                                                                       # skipped
    ]
    rec = _sampler_with(tmp_path, rows).stop()
    assert rec["samples"] == 3
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]


def test_clock_record_flags_slowdowns(tmp_path):
    rows = [
        "0, 1500, 2070, 1200.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
        "0, 1400, 2070, 1200.0, 0x0000000000000020, Not Active, Active, Active, Not Active",
    ]
    rec = _sampler_with(tmp_path, rows).stop()
    assert rec["sm_mhz"] == 1500.0
    assert rec["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_record_without_samples(tmp_path):
    rec = _sampler_with(tmp_path, ["", "nothing here"]).stop()
    assert rec["sm_mhz"] is None and rec["reasons"] == ["no samples"]


def test_scanned_pairs_counts_probed_list_lengths():
    offsets = np.array([0, 3, 3, 10, 12])          # list lengths 3, 0, 7, 2
    probes = np.array([[2, 0], [3, 2], [1, 0]])
    assert bench.scanned_pairs(offsets, probes) == (7 + 3) + (2 + 7) + (0 + 3)
