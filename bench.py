"""Benchmark of the three-species KLB hot path on GB300.

Default workload: the D3Q19 FP32 nanotube (512 x 128 x 128 box, staircase
pipe of radius 48, 6-cell solid shell, seeded couplings).  One benchmark step
is one check interval of the solver: 100 fused lattice steps (stream +
collide + interface coupling of water, electrons and phonons) followed by
the FP64 observation pass (flow rate, slip length, masses, momenta,
residual).

Other workloads (--workload):
  nanotube_noise  the default nanotube with thermal fluctuations of the
      water (kT = 1e-5, Philox-keyed noise after every collision).
  nanotube_large_{fp32,fp16,bf16}  the nanotube scaled to 768 x 192 x 192
      (radius 72, shell 9), populations in FP32 or as 16-bit differences
      from per-row references; same step as the default.
  sweep_{fp32,fp16}  96 seeded channels of a design sweep in one batch (one
      launch per lattice step, graph replay, autotuned block width; --scale
      multiplies every channel length); one
      benchmark step = 384 lattice steps of every channel + the observation
      pass of every channel.
  serving_{fp32,fp16}  a seeded Poisson stream of design-sweep requests
      (--rate per second, default 50) replayed against the request loop
      (--steps = requests); reports aggregate MLUPS and p50/p99 time to
      solution.
  design_map  pipes of radius 8..48 x water-electron couplings -0.02..0.05
      run to steady state through the request loop; reports aggregate MLUPS
      and the map of slip length, flow enhancement and electron wind.

Metric: MLUPS = active lattice sites (fluid + solid cells) updated per
second, whole job.  With N GPUs (torchrun) every rank runs its own replica
(independent channels of a design sweep: weak scaling, no data exchange).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload NAME]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LATTICE_STEPS_PER_STEP = 100
PROFILE = os.path.join(ROOT, "profiles", "k_step_d3q19_fp32_nanotube_512x128x128.md")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_source_hash():
    h = hashlib.sha256()
    for f in ("klb_kernels.cuh", "klb_step_pair.cuh", "klb_internal.h"):
        with open(os.path.join(ROOT, "paper_2403_15768_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic():
    """DRAM bytes per step-kernel launch from the committed ncu summary, if it
    was taken on the current kernel source; else None."""
    try:
        txt = open(PROFILE).read()
    except OSError:
        return None
    m_hash = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    m_b = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not (m_hash and m_b) or m_hash.group(1) != _kernel_source_hash():
        return None
    return float(m_b.group(1))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k] == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": rows[0][1],
                "reasons": reasons, "samples": len(rows)}


def _allreduce(dist, values, op, device):
    """Combine per-rank floats across ranks ("max": the slowest rank's time;
    "sum": work of all ranks); identity without a process group."""
    if dist is None:
        return [float(v) for v in values]
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return [float(v) for v in t]


def _dist_setup(gpus):
    import torch
    if gpus > 1 or "RANK" in os.environ:
        import torch.distributed as dist
        rank = int(os.environ.get("RANK", 0))
        local = int(os.environ.get("LOCAL_RANK", 0))
        world = int(os.environ.get("WORLD_SIZE", 1))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        return rank, local, world, dist
    return 0, 0, 1, None


def _oracle_workload(w) -> dict:
    return {"ny": w.ny, "nz": w.nz, "radius": w.radius, "shell": w.shell, "tau": list(w.tau),
            "rho0": w.rho0, "G": list(w.G), "couplings": list(w.couplings)}


def _slice_nx(w, procs):
    """x planes per oracle process: the box's planes shared out over the
    processes, so that together they hold the whole workload (the geometry
    is x-invariant and periodic in x, so a slice of nx planes does the
    per-site work of the full box)."""
    return max(1, -(-w.nx // procs))


def _cpu_baseline(w, seconds=10.0):
    """The FP64 oracle as it stands on the same workload, cut into one
    periodic x-slice per host core (single-threaded processes timing one
    common window; rates add), bounded to a window of `seconds`."""
    from oracle import throughput

    procs = os.cpu_count() or 1
    nx = _slice_nx(w, procs)
    res = throughput.run(_oracle_workload(w), procs, nx=nx, per=5, seconds=seconds)
    v = throughput.aggregate_mlups(res)
    n = sum(r["lattice_steps"] for r in res)
    return {"value": v, "unit": "MLUPS", "cores": procs, "kind": "oracle",
            "per_core": v / procs, "host": throughput.host_description(),
            "sample": f"the {w.nx}x{w.ny}x{w.nz} nanotube (r={w.radius}, shell {w.shell}) cut into "
                      f"{procs} periodic x-slices of {nx} planes, one single-threaded FP64 oracle per "
                      f"core ({n} lattice steps in total) over a common {seconds:.0f} s window"}


def run_reference(args):
    """The CPU oracle timed as the reference arm on the benchmark's own
    workload: the 512x128x128 nanotube cut into one periodic x-slice per host
    core (single-threaded processes, rates added over a common window); each
    step is 10 oracle lattice steps of every slice."""
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    from oracle import throughput
    from paper_2403_15768_gb300 import inputs

    w = inputs.PIPE_D3Q19_FP32
    procs = os.cpu_count() or 1
    nx, per = _slice_nx(w, procs), 10
    res = throughput.run(_oracle_workload(w), procs, nx=nx, per=per, steps=args.steps, warmup=args.warmup)
    v = throughput.aggregate_mlups(res)
    dt = max(r["seconds"] for r in res)
    line = {
        "impl": "reference", "metric": "MLUPS", "value": v, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "slice_nx": nx, "slices": procs, "lattice_steps_per_step": per,
                   "processes": procs},
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": procs, "kind": "oracle",
                         "host": throughput.host_description(),
                         "sample": f"the {w.nx}x{w.ny}x{w.nz} nanotube cut into {procs} periodic x-slices "
                                   f"of {nx} planes, {per} lattice steps per step in each of {procs} "
                                   f"single-threaded oracle processes"},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


STORAGE_BYTES = {"fp32": 4, "fp16": 2, "bf16": 2, "fp64": 8}
NOISE_KT = 1e-5  # thermal energy of the nanotube_noise workload (lattice units)


def _step_launch_ms(lat, stream, blocks, warmup=2):
    """Mean time per step-kernel launch: CUDA events on the lattice's stream
    around blocks of LATTICE_STEPS_PER_STEP steps (an observation pass after
    each block, outside the events), after warm-up blocks."""
    import torch

    for _ in range(warmup):
        lat.step(LATTICE_STEPS_PER_STEP)
        lat.observables()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(blocks)]
    torch.cuda.synchronize()
    for a, b in ev:
        a.record(stream)
        lat.step(LATTICE_STEPS_PER_STEP)
        b.record(stream)
        lat.observables()
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / (blocks * LATTICE_STEPS_PER_STEP)


def _precision_block(dev, blocks=5):
    """FP32 against 16-bit storage on the 768 x 192 x 192 nanotube (radius 72,
    shell 9): per storage the step kernel's launch time, its site rate and
    its fraction of the measured HBM bandwidth, and the 16-bit / FP32
    ratios of the cell rate."""
    import torch

    from paper_2403_15768_gb300 import inputs, klb

    peak, _ = _peaks()
    out = {"workload": inputs.PIPE_D3Q19_LARGE.name, "timing": f"CUDA events around {blocks} blocks "
           f"of {LATTICE_STEPS_PER_STEP} steps after 2 warm-up blocks"}
    for storage in ("fp32", "fp16", "bf16"):
        w = inputs.PIPE_D3Q19_LARGE.with_(storage=storage)
        stream = torch.cuda.Stream(dev)
        with torch.cuda.stream(stream):
            lat = klb.lattice_from_workload(w, device=dev, stream=stream)
            ms = _step_launch_ms(lat, stream, blocks)
            sites = lat.active_sites()
            cells = sum(lat.species_cells(s) for s in range(3))
            lat.close()
        nbytes = cells * 2 * 19 * STORAGE_BYTES[storage]
        out[storage] = {"launch_ms": ms, "mlups": sites / (ms * 1e-3) / 1e6,
                        "bytes_per_launch": nbytes,
                        "roofline_frac": nbytes / (ms * 1e-3) / 1e9 / peak}
        del lat
        torch.cuda.empty_cache()
    for storage in ("fp16", "bf16"):
        out[f"{storage}_over_fp32"] = out[storage]["mlups"] / out["fp32"]["mlups"]
    return out


def _serving_block(dev, n=12):
    """A short seeded trace of the request loop per storage (n requests of
    the Poisson stream, 50 per second, seed 0, cells log-uniform in
    [32^3, 512 x 128 x 128], run to the residual tolerance or 2 x 10^4
    steps; the batch block width autotuned at every re-forming of the
    batch): p50 / p99 time to solution and aggregate MLUPS."""
    import torch

    from paper_2403_15768_gb300 import inputs, klb, serving

    out = {"requests": n, "rate_per_s": 50.0, "max_steps": 20000, "check_every": 100, "autotune_steps": 5}
    for storage in ("fp32", "fp16"):
        tol = 1e-9 if storage == "fp32" else 1e-7
        stream = torch.cuda.Stream(dev)
        with torch.cuda.stream(stream):
            srv = klb.Server(40 * 10 ** 9, storage=storage, check_every=100, max_resident=128,
                             autotune_steps=5, device=dev, stream=stream)
            serving.replay(srv, inputs.request_stream(2, rate=50.0, seed=1000, storage=storage,
                                                      max_cells=64 ** 3), tol=tol, max_steps=1000)
            run = serving.replay(srv, inputs.request_stream(n, rate=50.0, seed=0, storage=storage),
                                 tol=tol, max_steps=20000)
            srv.close()
            del srv
        summ = serving.summarise(run)
        out[storage] = {"mlups": summ["site_updates"] / summ["makespan_s"] / 1e6, "tol": tol,
                        **{k: summ[k] for k in ("p50_s", "p99_s", "makespan_s", "status")}}
        torch.cuda.empty_cache()
    out["fp16_over_fp32"] = out["fp16"]["mlups"] / out["fp32"]["mlups"]
    return out


def run(args):
    if args.workload.startswith("sweep_"):
        return run_sweep(args)
    if args.workload.startswith("serving_"):
        return run_serving(args)
    if args.workload == "design_map":
        return run_design_map(args)
    import torch

    from paper_2403_15768_gb300 import inputs, klb

    rank, local, world, dist = _dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    kT = NOISE_KT if args.workload == "nanotube_noise" else 0.0
    if args.workload in ("nanotube", "nanotube_noise"):
        w = inputs.PIPE_D3Q19_FP32
    else:
        w = inputs.PIPE_D3Q19_LARGE.with_(storage=args.workload.rsplit("_", 1)[1])
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        lat = klb.lattice_from_workload(w, device=dev, stream=stream)
        if kT > 0.0:
            lat.set_fluctuations(kT, seed=rank)
    sites = lat.active_sites()
    species_cells = sum(lat.species_cells(s) for s in range(3))
    bytes_per_launch = species_cells * 2 * 19 * STORAGE_BYTES[w.storage]  # read + write of every population

    def interval():
        lat.step(LATTICE_STEPS_PER_STEP)
        return lat.observables()

    for _ in range(args.warmup):
        interval()
    torch.cuda.synchronize(dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # ---- device-timed region: inputs resident in HBM
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        t_start.record(stream)
        for k in range(args.steps):
            ev[k][0].record(stream)
            lat.step(LATTICE_STEPS_PER_STEP)
            ev[k][1].record(stream)
            obs = lat.observables()
        t_end.record(stream)
        barrier()
    ms = t_start.elapsed_time(t_end)
    step_kernel_ms = sum(a.elapsed_time(b) for a, b in ev) / (args.steps * LATTICE_STEPS_PER_STEP)

    # ---- end to end through the C ABI: couplings from pinned host memory,
    # 100 steps, observables back to the host, every step.
    cp_host = torch.tensor(w.couplings, dtype=torch.float64).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        lat.set_couplings(*cp_host.tolist())
        lat.step(LATTICE_STEPS_PER_STEP)
        obs_e2e = lat.observables()
    barrier()
    e2e_s = time.perf_counter() - t0

    ms, e2e_ms = _allreduce(dist, [ms, e2e_s * 1e3], "max", dev)

    if rank != 0:
        return
    lattice_updates = sites * LATTICE_STEPS_PER_STEP * args.steps * world
    value = lattice_updates / (ms * 1e-3) / 1e6
    e2e_value = lattice_updates / (e2e_ms * 1e-3) / 1e6
    peak, peak_kind = _peaks()
    achieved = bytes_per_launch / (step_kernel_ms * 1e-3) / 1e9
    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w.name, "lattice": "D3Q19", "storage": w.storage,
                   "box": [w.nx, w.ny, w.nz],
                   "radius": w.radius, "shell": w.shell, "active_sites": sites,
                   "species_cells": species_cells,
                   "lattice_steps_per_step": LATTICE_STEPS_PER_STEP,
                   "observables_per_step": 1, "parallelism": f"replicas x{world}",
                   "l2": f"working set {lat.nbytes / 1e9:.2f} GB per GPU > 129 MB L2, no flush needed",
                   "couplings": list(w.couplings), **({"kT": kT} if kT > 0 else {})},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": _ncu_traffic() if args.workload == "nanotube" else None,
                     "kernel": f"k_step<19,float,{w.storage}{',noise' if kT > 0 else ''}>",
                     "peak_source": peak_kind,
                     "bytes_per_launch": bytes_per_launch, "launch_ms": step_kernel_ms},
        "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": 40,
                "d2h_bytes_per_step": 144},
        "species_cell_updates": {"value": value * species_cells / sites, "unit": "M species-cells/s"},
        "gpu_launches": args.steps * (LATTICE_STEPS_PER_STEP + 2),
        "clocks": clk.summary(),
        "observables": {"flow_rate": obs["flow_rate"], "slip_length": obs["slip_length"],
                        "step": obs["step"], "e2e_step": obs_e2e["step"]},
    }
    if args.workload == "nanotube" and not args.no_extras:
        lat.close()
        del lat
        torch.cuda.empty_cache()
        line["precision"] = _precision_block(dev)
        line["serving"] = _serving_block(dev)
    if world == 1:
        line["cpu_baseline"] = _cpu_baseline(w)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


SWEEP_STEPS = 384  # lattice steps per benchmark step of a sweep: one 16-bit period


def _sweep_bytes(lats, storage):
    return sum(sum(l.species_cells(s) for s in range(3)) for l in lats) * 2 * 19 * STORAGE_BYTES[storage]


def run_sweep(args):
    """96 channels of a design sweep advanced as one batch."""
    import torch

    from paper_2403_15768_gb300 import inputs, klb

    rank, local, world, dist = _dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    storage = args.workload.split("_", 1)[1]
    ws = inputs.channel_sweep(96, seed=rank, storage=storage, scale=args.scale)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        lats = [klb.lattice_from_workload(w, device=dev, stream=stream) for w in ws]
        batch = klb.Batch(lats)
        width = batch.autotune(steps_per_candidate=8)
    sites = sum(l.active_sites() for l in lats)
    bytes_per_launch = _sweep_bytes(lats, storage)

    def interval():
        batch.step(SWEEP_STEPS)
        return [l.observables() for l in lats]

    with torch.cuda.stream(stream):
        batch.step((-lats[0].nstep) % SWEEP_STEPS)  # start the timed steps at a period boundary
        for _ in range(args.warmup):
            interval()
    torch.cuda.synchronize(dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk, torch.cuda.stream(stream):
        barrier()
        t_start.record(stream)
        for k in range(args.steps):
            ev[k][0].record(stream)
            batch.step(SWEEP_STEPS)
            ev[k][1].record(stream)
            obs = [l.observables() for l in lats]
        t_end.record(stream)
        barrier()
    ms = t_start.elapsed_time(t_end)
    step_ms = sum(a.elapsed_time(b) for a, b in ev) / (args.steps * SWEEP_STEPS)

    cp_host = [torch.tensor(w.couplings, dtype=torch.float64).pin_memory() for w in ws]
    with torch.cuda.stream(stream):
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for l, c in zip(lats, cp_host):
                l.set_couplings(*c.tolist())
            batch.step(SWEEP_STEPS)
            obs_e2e = [l.observables() for l in lats]
        barrier()
    e2e_ms = (time.perf_counter() - t0) * 1e3
    ms, e2e_ms = _allreduce(dist, [ms, e2e_ms], "max", dev)
    if rank != 0:
        return
    updates = sites * SWEEP_STEPS * args.steps * world
    peak, peak_kind = _peaks()
    achieved = bytes_per_launch / (step_ms * 1e-3) / 1e9
    line = {
        "metric": "MLUPS", "value": updates / (ms * 1e-3) / 1e6, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"design sweep of 96 D3Q19 channels (seed = rank), {storage}"
                               + (f", lengths x{args.scale:g}" if args.scale != 1.0 else ""),
                   "storage": storage, "channels": len(lats), "active_sites": sites,
                   "lattice_steps_per_step": SWEEP_STEPS, "block_width": width,
                   "blocks_per_launch": batch.blocks, "parallelism": f"replicas x{world}",
                   "l2": f"working set {sum(l.nbytes for l in lats) / 1e9:.1f} GB > 129 MB L2, no flush needed"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": f"k_step_batch<19,float,{storage}>", "peak_source": peak_kind,
                     "bytes_per_launch": bytes_per_launch, "launch_ms": step_ms},
        "e2e": {"value": updates / (e2e_ms * 1e-3) / 1e6, "unit": "MLUPS",
                "h2d_bytes_per_step": 40 * len(lats), "d2h_bytes_per_step": 144 * len(lats)},
        "gpu_launches": args.steps * (SWEEP_STEPS + 2 * len(lats) +
                                      (2 * len(lats) * SWEEP_STEPS // 32 if storage != "fp32" else 0)),
        "clocks": clk.summary(),
        "observables": {"flow_rate_first3": [o["flow_rate"] for o in obs[:3]],
                        "e2e_step": obs_e2e[0]["step"]},
    }
    if world == 1:
        line["cpu_baseline"] = _cpu_baseline(inputs.PIPE_D3Q19_FP32)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_serving(args):
    """A Poisson stream of design-sweep requests (50 per second, seeded)
    replayed against the request loop; --steps requests, --warmup requests
    of a warm-up replay."""
    import torch

    from paper_2403_15768_gb300 import inputs, klb, serving

    rank, local, world, dist = _dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    storage = args.workload.split("_", 1)[1]
    tol = 1e-9 if storage == "fp32" else 1e-7
    max_steps = 20000
    arena = 150 * 10 ** 9
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        srv = klb.Server(arena, storage=storage, check_every=100, max_resident=128, autotune_steps=5,
                         device=dev, stream=stream)
        if args.warmup:
            warm = inputs.request_stream(args.warmup, rate=50.0, seed=1000 + rank, storage=storage,
                                         max_cells=64 ** 3)
            serving.replay(srv, warm, tol=tol, max_steps=2000)
        reqs = inputs.request_stream(args.steps, rate=args.rate, seed=rank, storage=storage)
        with ClockSampler(local) as clk:
            run = serving.replay(srv, reqs, tol=tol, max_steps=max_steps)
    summ = serving.summarise(run)
    srv.close()
    summ["makespan_s"] = _allreduce(dist, [summ["makespan_s"]], "max", dev)[0]
    summ["site_updates"] = _allreduce(dist, [summ["site_updates"]], "sum", dev)[0]
    if rank != 0:
        return
    value = summ["site_updates"] / summ["makespan_s"] / 1e6
    res = [r for r in run["results"] if r]
    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * summ["makespan_s"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"Poisson request stream, {args.rate:g}/s, seed = rank, {storage}",
                   "rate_per_s": args.rate,
                   "storage": storage, "requests": args.steps, "tol": tol, "max_steps": max_steps,
                   "check_every": 100, "autotune_steps": 5, "arena_bytes": arena,
                   "parallelism": f"replicas x{world}"},
        "serving": {k: summ[k] for k in ("p50_s", "p99_s", "mean_s", "wait_p50_s", "wait_p99_s",
                                          "status", "makespan_s")},
        "roofline": None,
        "e2e": {"value": value, "unit": "MLUPS",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                "note": "requests enter and results leave through the host API; the makespan is host wall time"},
        "gpu_launches": int(run["stats"]["rounds"] * 100),
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_design_map(args):
    """A design map of the nanotube permeability study's shape: pipes of
    radius 8..48 for water-electron couplings -0.02 .. 0.05 (negative quantum
    friction included), each run from rest to steady state through the
    request loop; reports aggregate MLUPS and the map."""
    import torch

    from paper_2403_15768_gb300 import inputs, klb, serving

    rank, local, world, dist = _dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ws = inputs.design_grid(range(8, 49, 8), [-0.02, 0.0, 0.02, 0.05])
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        srv = klb.Server(32 * 10 ** 9, storage="fp32", check_every=200, max_resident=64, device=dev,
                         stream=stream)
        serving.design_map(srv, ws[:2], tol=1e-6, max_steps=400)  # warm-up
        with ClockSampler(local) as clk:
            t0 = time.perf_counter()
            res = serving.design_map(srv, ws, tol=1e-9, max_steps=100_000)
            wall = time.perf_counter() - t0
        rounds = srv.stats()["rounds"]
        srv.close()
    updates = float(sum(r["sites"] * r["steps"] for r in res))
    wall = _allreduce(dist, [wall], "max", dev)[0]
    updates = _allreduce(dist, [updates], "sum", dev)[0]
    if rank != 0:
        return
    value = updates / wall / 1e6
    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": len(ws),
        "warmup": 2, "ms_per_step": 1e3 * wall / len(ws), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "design map: D3Q19 pipes R = 8..48 x g_we = -0.02..0.05, FP32, tol 1e-9",
                   "requests": len(ws), "parallelism": f"replicas x{world}"},
        "map": [[r["radius"], r["g_we"], r["slip_length"], r["enhancement"], r["mean_u_e"], r["steps"],
                 r["status"]] for r in res],
        "roofline": None,
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                "note": "requests enter and results leave through the host API; wall time"},
        "gpu_launches": int(rounds * 200),
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


WORKLOADS = ["nanotube", "nanotube_noise", "nanotube_large_fp32", "nanotube_large_fp16", "nanotube_large_bf16",
             "sweep_fp32", "sweep_fp16", "serving_fp32", "serving_fp16", "design_map"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="nanotube", choices=WORKLOADS)
    ap.add_argument("--rate", type=float, default=50.0, help="serving: requests per second")
    ap.add_argument("--no-extras", dest="no_extras", action="store_true",
                    help="default workload: leave out the precision and serving blocks")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="sweeps: every channel length times this factor (1 = the 96-channel sweep)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 48 if args.workload.startswith("serving_") else (
            4 if args.workload.startswith("sweep_") else 20)
    if args.impl == "reference":
        run_reference(args)
    else:
        run(args)


if __name__ == "__main__":
    main()
