"""The reference arm of bench.py (the FP64 oracle on the host cores) prints
one JSON line with the contract's keys and the GB300 arm's workload config.
Runs on the CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"]
    assert line["config"]["workload"] == "x4_adaptive_31^4->81^4_weno5_update"
    assert line["config"]["grid_fine"] == [81, 81, 81, 81]
    assert line["config"]["grid_coarse"] == [31, 31, 31, 31]
    # the same config dict as the GB300 arm's line; the sample is described
    # under cpu_baseline
    import bench
    assert line["config"] == json.loads(json.dumps(bench.arm_config()))
    assert "TVD-RK3 step" in line["cpu_baseline"]["sample"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["unit"] == line["unit"]
