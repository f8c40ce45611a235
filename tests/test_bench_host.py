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
    workload at bounded sizes (a few to some tens of seconds of oracle work)."""
    name, mats = bench.medium_workload()
    for small in (True, False):
        sname, smats = bench.cpu_sample(small)
        assert [cfg for _, cfg in smats] == [cfg for _, cfg in mats]
        assert sum(A.nnz for A, _ in smats) < 0.1 * sum(A.nnz for A, _ in mats)
        assert sname != name


def test_owner_parts_from_tree():
    """Owners for the cut metrics: a leaf owns its range, a split node owns
    its separator, placed last (BBD) or between the parts (SBD)."""
    import numpy as np
    import torch
    perm = np.array([5, 3, 1, 0, 4, 2, 6], dtype=np.int32)
    # root: 7 vertices, n1 = 3, n2 = 2, nsep = 2; children leaves
    for sbd in (False, True):
        off = [0, 0, 5 if sbd else 3]
        tree = {"offset": torch.tensor(off), "n1": torch.tensor([3, 3, 2]), "n2": torch.tensor([2, 0, 0]),
                "nsep": torch.tensor([2, 0, 0])}
        if sbd:
            tree["offset"] = torch.tensor([0, 0, 5])
        part = bench.owner_parts(7, perm, tree, sbd)
        sep = perm[3:5] if sbd else perm[5:7]
        assert sorted(np.flatnonzero(part == 0).tolist()) == sorted(sep.tolist())
        assert sorted(np.flatnonzero(part == 1).tolist()) == sorted(perm[0:3].tolist())
        assert (part >= 0).all()


def test_host_cpu_reports_model_and_cores():
    h = bench.host_cpu()
    assert h["cpu_cores"] >= 1 and isinstance(h["cpu_model"], str) and h["arch"]
