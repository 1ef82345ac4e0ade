"""Host-side parts of the benchmark, without a GPU: the summary of the clock
samples taken during a timed region (median SM clock, the highest maximum
clock, every throttle reason seen active) and the workload description both
arms print."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
from paper_2410_16727_gb300 import inputs as I  # noqa: E402

# index, clocks.sm, clocks.max.sm, power.draw, reasons bitmask, hw_slowdown,
# hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap (csv, noheader, nounits)
ROWS = [
    "0, 2070, 2070, 910.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "0, 2055, 2070, 1290.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
    "0, 2040, 2070, 1391.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
    "0, [N/A], 2070, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",
    "garbage line",
]


def _sampler(tmp_path, lines):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    s.proc = object()          # as if nvidia-smi had run
    return s


def test_clock_summary_median_max_and_reasons(tmp_path):
    out = _sampler(tmp_path, ROWS).summary()
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["samples"] == 4


def test_clock_summary_reports_each_slowdown(tmp_path):
    rows = ["0, 1500, 2070, 800, 0x8, Active, Not Active, Active, Not Active",
            "0, 1600, 2070, 800, 0x40, Not Active, Active, Not Active, Not Active"]
    out = _sampler(tmp_path, rows).summary()
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1550.0


def test_clock_summary_without_samples(tmp_path):
    assert _sampler(tmp_path, ["garbage"]).summary()["reasons"] == ["no samples"]
    s = bench.ClockSampler(0)
    assert s.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_workload_config_names_the_stress_workload():
    cfg = bench.workload_config(I.WORKLOADS["stress"], 1)
    assert cfg["workload"].startswith("stress: 1024 problems x 128 seeds x 64 waypoints, 200 L-BFGS iterations, "
                                      "16 clutter scenes, ESDF 256^3 at 5 mm")
    assert (cfg["problems"], cfg["seeds"], cfg["waypoints"], cfg["iters"]) == (1024, 128, 64, 200)
    assert cfg["parallelism"] == "replicas x1"
