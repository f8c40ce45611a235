"""Host-side logic of bench.py that needs no GPU: the clock record that decides
whether a timed run stands (median SM clock under load, throttle reasons),
and the bounded oracle samples of the reference arm and the CPU baselines."""
import os

import bench


def _clocks_file(tmp_path, rows):
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(rows) + "\n")
    c = bench.ClockSampler(0)
    c.proc = object()  # as if nvidia-smi had been started
    c.path = str(p)
    return c


def test_clock_summary_median_and_reasons(tmp_path):
    rows = ["0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
            "garbage line"]
    s = _clocks_file(tmp_path, rows).summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_slowdown(tmp_path):
    rows = ["0, 1500, 2070, 1380.0, 0x20, Not Active, Active, Not Active, Not Active",
            "0, 1400, 2070, 1390.0, 0x40, Active, Not Active, Active, Not Active"]
    s = _clocks_file(tmp_path, rows).summary()
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert s["sm_mhz"] == 1450.0


def test_clock_summary_without_sampler():
    c = bench.ClockSampler(0)
    assert c.summary() is None


def test_oracle_samples_are_bounded_versions_of_the_workload():
    """The CPU samples keep the two families and parameters of the medium
    workload at sizes the oracle finishes in seconds."""
    name, mats = bench.medium_workload()
    for small in (True, False):
        sname, smats = bench.cpu_sample(small)
        assert [cfg for _, cfg in smats] == [cfg for _, cfg in mats]
        assert sum(A.nnz for A, _ in smats) < 0.02 * sum(A.nnz for A, _ in mats)
        assert sname != name
