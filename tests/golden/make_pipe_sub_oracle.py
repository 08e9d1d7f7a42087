"""Writes tests/golden/pipe_sub_perturbed_5000.npz: the FP64 oracle's result
for the 128 x 64 x 64 nanotube subcase (radius 24, shell 3; the nanotube
of Sec. 5.1 at half the benchmark's scale) after 5000 steps from a seeded,
x-varying perturbed start (inputs.perturbation, seed 5, eps 1e-3).

The oracle needs about ten minutes of one CPU core for this run, too long
for every GPU test session, so its result is stored: every observable (flow
rate, slip fit, wall-row and species means, masses, momenta) and the density
and velocity fields of all species on the x planes listed in PLANES.  Only
oracle/ computes anything here; the inputs come from the seeded input module.

    python tests/golden/make_pipe_sub_oracle.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import Oracle, cross_section, observables_from_fields  # noqa: E402
from paper_2403_15768_gb300 import inputs  # noqa: E402

STEPS = 5000
SEED, EPS = 5, 1e-3
PLANES = (0, 45, 90)
OUT = os.path.join(HERE, "pipe_sub_perturbed_5000.npz")


def main():
    w = inputs.PIPE_D3Q19_SUB
    geo = cross_section("pipe", w.ny, w.nz, radius=w.radius, shell=w.shell)
    o = Oracle(w.kind, w.nx, geo, tau=w.tau, rho0=w.rho0, G=w.G, couplings=w.couplings)
    drho, u = inputs.perturbation(w, SEED, EPS)
    o.init_equilibrium(drho, u)
    o.step(STEPS)
    f = o.observe()
    ob = observables_from_fields(geo, w.nx, w.rho0, f)
    planes = np.array(PLANES)
    np.savez_compressed(OUT, steps=STEPS, seed=SEED, eps=EPS, planes=planes,
                        u=f["u"][..., planes], drho=f["drho"][..., planes],
                        observables=json.dumps(ob))
    print(OUT, json.dumps(ob))


if __name__ == "__main__":
    main()
