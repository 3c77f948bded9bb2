"""The benchmark's reference arm (the CPU oracle on a bounded sample) prints
one JSON line with the keys of the GPU arm's line, on the GPU arm's metric,
unit, direction and workload config; the clock sampler's parser."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--cpu-queries", "1"], cwd=ROOT, capture_output=True,
                         text=True, timeout=600, check=True).stdout.strip().splitlines()
    assert len(out) == 1
    line = json.loads(out[0])
    sys.path.insert(0, ROOT)
    import bench
    assert line["impl"] == "reference"
    assert (line["metric"], line["unit"], line["higher_is_better"]) == (bench.METRIC, bench.UNIT,
                                                                        True)
    assert line["config"] == bench._star_config(line["config"]["queries"], 1, 1)
    assert line["n_gpus"] == 1 and line["steps"] == 1 and line["warmup"] == 3
    assert line["value"] > 0 and line["ms_per_step"] > 0 and line["vs_baseline"] is None
    assert line["scaling"] == "weak" and line["dtype"] == "f64"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["unit"] == line["unit"]
    assert cb["cores"] >= 1 and "1 of the" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_clock_samples_summary():
    """The nvidia-smi sampler's parser: median SM clock, the maximum, and
    every throttle reason seen Active in any sample; "[N/A]" or short lines
    are skipped."""
    sys.path.insert(0, ROOT)
    import bench
    c = bench.Clocks(0)
    c.out = "\n".join([
        "0, 2070 MHz, 2070 MHz, 900.10 W, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980 MHz, 2070 MHz, 1390.00 W, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2055 MHz, 2070 MHz, 1200.00 W, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070 MHz, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",
        "0, 2070 MHz",
    ])
    s = c.summary()
    assert s == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.out = "0, 2070 MHz, 2070 MHz, 900 W, 0x0, Active, Not Active, Active, Not Active"
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    c.out = ""
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
