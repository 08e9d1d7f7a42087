"""Site-update rate of the FP64 oracle on a bounded sample of a pipe workload,
on all host cores.

TEST INFRASTRUCTURE ONLY: used by the CPU-baseline leg of ``bench.py``.  The
oracle runs as it stands (single-threaded C): the host's cores are used by
running one independent sample per process, all processes timing the same
wall-clock window, and the rates are added.  The sample is the workload's
full cross-section with a few x planes; the geometry is x-invariant, so the
per-site work equals that of the full box.

Run as ``python -m oracle.throughput '<json spec>'`` (one sample; prints one
JSON line), or call :func:`run` to start ``procs`` such processes.
"""
import json
import os
import platform
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def host_description() -> str:
    """CPU model and logical core count of this host."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return f"{model or platform.machine()}, nproc {os.cpu_count()}"


def _sample(w, nx):
    from oracle import Oracle, cross_section

    geo = cross_section("pipe", w["ny"], w["nz"], radius=w["radius"], shell=w["shell"])
    o = Oracle(19, nx, geo, tau=tuple(w["tau"]), rho0=w["rho0"], G=tuple(w["G"]),
               couplings=tuple(w["couplings"]))
    o.init_equilibrium()
    sites = int(((geo.cs_type == 1) | (geo.cs_type == 2)).sum()) * nx
    return o, sites


def _child(spec):
    o, sites = _sample(spec["workload"], spec["nx"])
    o.step(2)
    per = spec["per"]
    for _ in range(spec["warmup"]):
        o.step(per)
    while time.time() < spec["start"]:
        time.sleep(0.0005)
    n, t0 = 0, time.perf_counter()
    if spec["steps"] > 0:
        for _ in range(spec["steps"]):
            o.step(per)
            n += per
    else:
        while time.perf_counter() - t0 < spec["seconds"]:
            o.step(per)
            n += per
    dt = time.perf_counter() - t0
    print(json.dumps({"site_updates": sites * n, "seconds": dt, "lattice_steps": n, "sites": sites}))


def run(workload: dict, procs: int, nx: int = 8, per: int = 5, seconds: float = 10.0,
        steps: int = 0, warmup: int = 0, start_delay: float = 4.0):
    """Start ``procs`` single-threaded oracle processes on the same sample.
    Each runs ``warmup`` untimed blocks of ``per`` lattice steps, waits for a
    common start time, then times ``steps`` blocks (or, with ``steps`` = 0,
    as many blocks as fit in ``seconds``).  Returns the per-process results."""
    spec = {"workload": workload, "nx": nx, "per": per, "seconds": seconds, "steps": steps,
            "warmup": warmup, "start": time.time() + start_delay}
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    children = [subprocess.Popen([sys.executable, "-m", "oracle.throughput", json.dumps(spec)], cwd=ROOT,
                                 env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
                for _ in range(procs)]
    out = []
    for c in children:
        so, se = c.communicate()
        if c.returncode != 0:
            raise RuntimeError(f"oracle sample process failed: {se.strip()[-500:]}")
        out.append(json.loads(so.strip().splitlines()[-1]))
    return out


def aggregate_mlups(results) -> float:
    """Sum of the processes' rates over their common window."""
    return sum(r["site_updates"] / r["seconds"] for r in results) / 1e6


if __name__ == "__main__":
    _child(json.loads(sys.argv[1]))
