"""bench.py's command-line contract, on CPU.

- `--impl reference` times the float64 oracle on the host cores and prints one JSON line with the
  keys a driver reads: the metric, its unit and direction, whole-job value, an `e2e` object with
  zero copy bytes (nothing crosses PCIe), and a `cpu_baseline` stating what was timed.
- The GPU arm never falls back to the CPU: without a CUDA device it exits with an error and
  prints no result line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args, timeout=600):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_json_line():
    r = _run("--impl", "reference", "--steps", "1", "--warmup", "0", "--workload", "mid", "--views", "2",
             "--band-rows", "2")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference"
    assert out["unit"] == "contribs/s" and out["higher_is_better"] is True
    assert out["value"] > 0 and out["steps"] == 1 and out["warmup"] == 0 and out["n_gpus"] == 1
    assert out["config"]["views"] == 2 and "workload" in out["config"]
    e2e = out["e2e"]
    assert e2e["value"] == out["value"] and e2e["unit"] == out["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    cpu = out["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == out["value"]
    assert "2 views of the 2" in cpu["sample"] and "tile rows" in cpu["sample"]


def test_gpu_arm_fails_loudly_without_cuda():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    r = _run("--steps", "1", "--warmup", "0", "--views", "1", "--no-cpu", "--no-forms", "--no-e2e")
    assert r.returncode != 0
    assert "cuda" in r.stderr.lower() or "nvidia" in r.stderr.lower(), r.stderr[-2000:]
    assert not any(l.strip().startswith("{") for l in r.stdout.splitlines())


def test_clock_record_summary():
    # nvidia-smi lines as the sampler reads them: sm, max sm, power, active mask, then the
    # hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown and sw_power_cap states
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler("0")
    c.lines = ["1965, 2032, 700.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
               "2032, 2032, 650.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
               "2010, 2032, 690.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
               "[N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",
               "not a sample"]
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2010.0 and s["sm_max_mhz"] == 2032.0
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = ["1400, 2032, 900.0, 0x0000000000000008, Active, Not Active, Active, Not Active"]
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    c.lines = []
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
