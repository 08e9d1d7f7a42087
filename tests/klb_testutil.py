"""Glue for the tests: build the oracle and the CUDA lattice of one workload.

The two sides share only the seeded inputs of ``paper_2403_15768_gb300.inputs``;
each builds its own geometry and does its own arithmetic.
"""
from __future__ import annotations

import numpy as np

from oracle import Oracle, cross_section
from paper_2403_15768_gb300.inputs import Workload


def oracle_geometry(w: Workload):
    if w.geom == "slab":
        return cross_section("slab", w.ny, w.nz, width=w.width, shell=w.shell)
    if w.geom == "pipe":
        return cross_section("pipe", w.ny, w.nz, radius=w.radius, shell=w.shell)
    return cross_section("mask", w.ny, w.nz, mask=w.extra["mask"],
                         periodic_y=w.extra.get("periodic_y", False),
                         periodic_z=w.extra.get("periodic_z", False))


def make_oracle(w: Workload, nx=None) -> Oracle:
    return Oracle(w.kind, nx or w.nx, oracle_geometry(w), tau=w.tau, rho0=w.rho0, G=w.G,
                  couplings=w.couplings, iface_bounceback=(w.iface_bc == "bounceback"),
                  phonon_wave=w.phonon_wave)


def species_masks(geo, nx):
    t = geo.cs_type
    fluid = np.broadcast_to((t == 1)[:, :, None], (geo.nz, geo.ny, nx))
    solid = np.broadcast_to((t == 2)[:, :, None], (geo.nz, geo.ny, nx))
    return [fluid, solid, solid]


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
