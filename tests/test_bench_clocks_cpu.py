"""The bench's clock record (sampled with nvidia-smi during the timed
region) parsed from a fake sample file: median SM clock, the maximum, and
which throttle reasons were ever active ("Not Active" is not active)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


def _clocks(lines, name):
    sys.path.insert(0, ROOT)
    import bench
    c = bench.Clocks(0)
    c.proc = True                       # as if the sampler had run
    os.makedirs(os.path.join(HERE, "_build"), exist_ok=True)
    c.path = os.path.join(HERE, "_build", name)
    with open(c.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    return c.summary()


def test_median_clock_and_active_reasons():
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1380.5, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = _clocks(rows, "clocks_a.csv")
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_thermal_and_hardware_slowdown_are_reported():
    rows = [
        "0, 1500, 2070, 1400.0, 0x8, Active, Not Active, Not Active, Not Active",
        "0, 1400, 2070, 1400.0, 0x20, Not Active, Active, Active, Not Active",
    ]
    s = _clocks(rows, "clocks_b.csv")
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert s["sm_mhz"] == 1500.0 and s["samples"] == 2


def test_no_samples():
    assert _clocks([], "clocks_c.csv")["reasons"] == ["no samples"]
