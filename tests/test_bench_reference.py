"""The benchmark's reference arm (the FP64 oracle on the host cores) prints one
JSON line with the keys of the benchmark contract; a tiny run on the CPU."""
import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(HERE, "..", "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1", "--workload", "tiny"],
                         capture_output=True, text=True, timeout=600, check=True).stdout
    line = json.loads(out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference"
    assert line["value"] > 0 and line["higher_is_better"] is True
    # the same config object as the GPU arm's line for this workload
    sys.path.insert(0, os.path.join(HERE, ".."))
    import bench
    from paper_2410_16727_gb300 import inputs as I
    assert line["config"] == bench.workload_config(I.WORKLOADS["tiny"], 1)
    # the step time is what one step measured: value x step time = one problem's evaluations
    spec = I.WORKLOADS["tiny"]
    assert abs(line["value"] * line["ms_per_step"] * 1e-3 - spec.S * spec.T * spec.iters) < 1e-6 * line["value"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
