"""The benchmark's JSON line keeps its contract: one line with the metric,
the device-timed value, the end-to-end value through the C ABI with its
host<->device bytes, the step kernel's roofline against the measured peak,
the timed oracle baseline, the clocks seen during the timed region, the
number of library kernels launched, and the FP32-vs-16-bit and serving
blocks."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_default_bench_line():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, "bench.py", "--steps", "6", "--warmup", "3"], cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["metric"] == "MLUPS" and d["unit"] == "MLUPS" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 6 and d["warmup"] == 3 and d["scaling"] == "weak"
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["data"] == "synthetic" and d["dtype"] == "f32"
    assert d["config"]["workload"] == "d3q19_fp32_pipe_512x128x128_r48"
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and rf["peak"] > 0
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-9 and 0.3 < rf["frac"] < 1.2
    assert rf["bytes_per_launch"] == 5_693_440 * 2 * 19 * 4
    assert rf["traffic"] is None or 0.9 * rf["bytes_per_launch"] < rf["traffic"] < 1.1 * rf["bytes_per_launch"]
    e = d["e2e"]
    assert e["unit"] == "MLUPS" and e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] >= 1 and cb["sample"]
    assert d["gpu_launches"] == 6 * (100 + 2)
    clk = d["clocks"]
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(clk)
    # FP32 against 16-bit storage on the 768x192x192 nanotube, and a short
    # serving trace per storage (the metric's FP32-vs-FP16 and p50/p99 parts)
    pr = d["precision"]
    for st in ("fp32", "fp16", "bf16"):
        assert pr[st]["launch_ms"] > 0 and 0.1 < pr[st]["roofline_frac"] < 1.2
        assert pr[st]["bytes_per_launch"] == 19_184_640 * 2 * 19 * (4 if st == "fp32" else 2)
    assert abs(pr["fp16_over_fp32"] - pr["fp16"]["mlups"] / pr["fp32"]["mlups"]) < 1e-9
    sv = d["serving"]
    for st in ("fp32", "fp16"):
        assert sv[st]["mlups"] > 0 and 0 < sv[st]["p50_s"] <= sv[st]["p99_s"]
        assert sum(sv[st]["status"].values()) == sv["requests"]
