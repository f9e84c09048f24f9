"""The benchmark's JSON line: the reference arm (the FP64 oracle on the host, CPU only) and, on a
GPU, the device arm on a small batch."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, timeout=600):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       timeout=timeout, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    d = run_bench("--impl", "reference", "--steps", "1", "--warmup", "1")
    assert d["impl"] == "reference" and d["unit"] == "cell-updates/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


@pytest.mark.gpu
def test_device_arm_line():
    pytest.importorskip("torch")
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    d = run_bench("--samples", "8", "--T", "0.01", "--steps", "1", "--warmup", "3", "--no-cpu-baseline")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "e2e", "roofline", "clocks", "gpu_launches"):
        assert k in d, k
    assert d["value"] > 0 and d["gpu_launches"] > 0 and d["config"]["workload"]
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and 0 < r["frac"] < 2 and "traffic" in r
    assert d["e2e"]["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert d["alu_roofline"]["bound"] == "alu" and 0 < d["alu_roofline"]["frac"] < 1
    assert set(d["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}
    w = run_bench("--workload", "sod1024_fp64", "--steps", "1", "--warmup", "3")
    assert w["config"]["workload"] == "sod1024_fp64" and w["value"] > 0
