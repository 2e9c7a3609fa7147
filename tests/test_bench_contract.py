"""The benchmark's output contract, on the CPU: the reference arm (the oracle
on the host cores) prints one JSON line with the keys the benchmark protocol
names, on the same metric and unit as the GPU arm, and the helpers that
attach the profiled DRAM traffic accept only a capture of the current
kernel source."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_prints_one_line_with_the_contract_keys():
    d = _run("--impl", "reference", "--workload", "torus10", "--steps", "3", "--warmup", "3")
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 3 and d["warmup"] == 3
    assert d["metric"] == "GOM trials/sec (plain parallel GOM, weighted Max-Cut)" and d["unit"] == "trials/s"
    assert d["higher_is_better"] is True and d["value"] > 0
    assert d["config"]["workload"] == "torus10"
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1


def test_warmup_below_three_is_refused():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--warmup", "2"],
                         cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert out.returncode != 0 and "--warmup must be >= 3" in out.stderr


def test_profiled_traffic_only_for_the_current_source():
    sys.path.insert(0, ROOT)
    import bench
    h = bench.kernel_source_hash()
    with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as fh:
        d = json.load(fh)
    for key, e in d.items():
        if key.startswith("_"):
            continue
        kernel, workload = key.split(":")
        got = bench.profiled_traffic(workload, kernel + " (any description)")
        assert got == (e["dram_bytes_per_launch"] if e["kernel_hash"] == h else None), key
    assert bench.profiled_traffic("no_such_workload", "k_run_bs") is None
