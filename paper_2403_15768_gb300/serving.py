"""Client side of the request loop: replays a stream of timed requests
against a klb.Server and summarises time to solution.

Scheduling, admission, batching and retirement all happen in the native
server (klb_server_*); this module only submits each request when its
arrival time comes on the server's clock, calls the scheduling rounds and
collects results.
"""
from __future__ import annotations

import time

import numpy as np

from . import klb


def replay(server: "klb.Server", requests, tol: float, max_steps: int, max_seconds: float = 0.0,
           wall_limit: float | None = None) -> dict:
    """Submit ``requests`` (inputs.Request) at their arrival times, run
    rounds until every one has finished, and return the results in request
    order with the server's counters.  ``wall_limit`` (s) stops submitting
    and running early (the unfinished are reported as such)."""
    reqs = sorted(requests, key=lambda r: r.arrival)
    t0 = server.clock()
    nxt = 0
    done = {}
    while len(done) < len(reqs):
        now = server.clock() - t0
        if wall_limit is not None and now > wall_limit:
            break
        while nxt < len(reqs) and reqs[nxt].arrival <= now:
            r = reqs[nxt]
            server.submit(klb.desc_from_workload(r.w), r.w.couplings, tol, max_steps, r.rid,
                          arrival=t0 + r.arrival, max_seconds=max_seconds)
            nxt += 1
        server.tick()
        for res in server.poll():
            done[res["id"]] = res
        st = server.stats()
        if st["resident"] == 0 and st["queued"] == 0 and nxt < len(reqs):
            time.sleep(max(0.0, min(0.01, reqs[nxt].arrival - (server.clock() - t0))))
    end = server.clock() - t0
    return {"results": [done.get(r.rid) for r in requests], "stats": server.stats(),
            "makespan": end, "t0": t0}


def summarise(run: dict) -> dict:
    """Latency percentiles (time from arrival to retirement, queueing
    included), admission waits and aggregate throughput of a replay."""
    res = [r for r in run["results"] if r is not None]
    if not res:
        return {"finished": 0}
    lat = np.array([r["finished"] - r["arrival"] for r in res])
    wait = np.array([r["admitted"] - r["arrival"] for r in res])
    updates = float(sum(r["sites"] * r["steps"] for r in res))
    first = min(r["arrival"] for r in res)
    last = max(r["finished"] for r in res)
    status = {}
    for r in res:
        k = klb.STATUS.get(r["status"], str(r["status"]))
        status[k] = status.get(k, 0) + 1
    return {"finished": len(res), "submitted": len(run["results"]),
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "wait_p50_s": float(np.percentile(wait, 50)),
            "wait_p99_s": float(np.percentile(wait, 99)),
            "mlups": updates / max(last - first, 1e-9) / 1e6, "site_updates": updates,
            "status": status, "makespan_s": last - first}


def design_map(server: "klb.Server", workloads, tol: float, max_steps: int) -> list:
    """Run every workload (a design grid, e.g. inputs.design_grid) from rest
    to its steady state through the request loop and return, per workload,
    the status, steps, slip length, flow rate per unit length, the flow
    enhancement over the no-slip Poiseuille flow of the same effective radius
    (pi G d_wall^4 / (8 rho0 nu)) and the mean electron and phonon
    velocities (the electron and phonon winds)."""
    for k, w in enumerate(workloads):
        server.submit(klb.desc_from_workload(w), w.couplings, tol, max_steps, k)
    done = {}
    while len(done) < len(workloads):
        server.tick()
        for res in server.poll():
            done[res["id"]] = res
    out = []
    for k, w in enumerate(workloads):
        r = done[k]
        o = r["obs"]
        nu = (w.tau[0] - 0.5) / 3.0
        q0 = np.pi * w.G[0] * o["d_wall"] ** 4 / (8.0 * w.rho0 * nu)
        out.append({"name": w.name, "radius": w.radius, "g_we": w.couplings[0], "status": r["status"],
                    "steps": r["steps"], "slip_length": o["slip_length"], "flow_rate": o["flow_rate"],
                    "enhancement": o["flow_rate"] / q0, "mean_u_e": o["mean_u"][1],
                    "mean_u_p": o["mean_u"][2], "sites": r["sites"]})
    return out
