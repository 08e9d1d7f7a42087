"""The CPU baseline of the benchmark: the oracle, unchanged, run as one
single-threaded process per core over a common window (oracle.throughput),
and the reference arm's JSON line built from it."""
import json
import os
import subprocess
import sys

from oracle import throughput
from paper_2403_15768_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _small():
    w = inputs.PIPE_D3Q19_SUB
    return {"ny": w.ny, "nz": w.nz, "radius": w.radius, "shell": w.shell, "tau": list(w.tau),
            "rho0": w.rho0, "G": list(w.G), "couplings": list(w.couplings)}


def test_processes_share_one_window_and_rates_add():
    res = throughput.run(_small(), 2, nx=4, per=2, steps=3, warmup=1, start_delay=2.0)
    assert len(res) == 2
    for r in res:
        assert r["lattice_steps"] == 6 and r["site_updates"] == 6 * r["sites"] and r["seconds"] > 0
    assert res[0]["sites"] == res[1]["sites"]
    v = throughput.aggregate_mlups(res)
    assert abs(v - sum(r["site_updates"] / r["seconds"] for r in res) / 1e6) < 1e-12
    assert "nproc" in throughput.host_description()


def test_reference_arm_line():
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == "MLUPS" and line["value"] > 0
    assert line["cpu_baseline"]["cores"] == (os.cpu_count() or 1)
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_profile_traffic_follows_the_kernel_sources(monkeypatch):
    """The benchmark reports the committed ncu traffic of the step kernel only
    for the kernel sources it was taken on, and then within a few percent of
    the algorithmic bytes (no re-reads); after a source change it reports
    none."""
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    txt = open(bench.PROFILE).read()
    assert "kernel_source_sha256_16:" in txt and "dram_bytes_per_launch:" in txt
    algorithmic = 5_693_440 * 2 * 19 * 4
    t = bench._ncu_traffic()
    assert t is None or 0.95 * algorithmic < t < 1.05 * algorithmic
    monkeypatch.setattr(bench, "_kernel_source_hash", lambda: "0" * 16)
    assert bench._ncu_traffic() is None


def test_clock_summary_parsing():
    """The clocks object of the benchmark line: median SM clock under load,
    the maximum clock, and every throttle reason seen active."""
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_mod2", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    c = bench.ClockSampler(0)
    c.out = ("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
             "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
             "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
             "garbage line\n")
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.out = ""
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
