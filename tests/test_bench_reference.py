"""bench.py --impl reference (the FP64 CPU oracle as the comparison arm) runs
on the CPU and prints one JSON line with the benchmark contract's keys."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    line = json.loads(res.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1 and line["warmup"] >= 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["metric"] == "forward+loglik evals/s" and line["config"]["workload"].startswith("forward-g30-f60-k200")


def test_layer_sweep_refuses_counts_outside_the_row_stride():
    """--layer-sweep is checked on the host before any device work: counts
    outside 1..10 (the workload's row stride) or non-integers end with a
    usage error."""
    for bad in ("0,4", "11", "x", ","):
        res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--layer-sweep", bad],
                             capture_output=True, text=True, timeout=120, cwd=ROOT)
        assert res.returncode == 2 and "--layer-sweep" in res.stderr, (bad, res.stderr[-500:])
