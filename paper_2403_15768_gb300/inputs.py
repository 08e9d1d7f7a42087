"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

Holds none of the method's arithmetic: named workload presets (sizes and
parameters of the nanochannel set-ups), the coupling draws and the random
numbers of perturbed starts.  Both the CUDA path and the CPU oracle take
these as inputs and compute everything else themselves.

The paper runs no simulation and names no dataset; its set-ups (Sec. 2,
Sec. 5.1: water driven through a carbon nanotube or a slab channel with
solid walls carrying electrons and phonons) are stood in for by these
synthetic channels.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    kind: int            # 9 (D2Q9) or 19 (D3Q19)
    geom: str            # "slab", "pipe" or "mask"
    nx: int
    ny: int
    nz: int
    width: int = 0       # slab fluid rows
    radius: int = 0      # pipe radius
    shell: int = 0       # solid thickness
    tau: tuple = (0.8, 0.6, 1.0)
    rho0: float = 1.0
    G: tuple = (1e-6, 0.0, 0.0)
    couplings: tuple = (0.0, 0.0, 0.0, 0.0, 0.0)  # g_we, g_wp, g_ep, g_ec, g_pc
    storage: str = "fp32"
    steps: int = 0
    iface_bc: str = "specular"
    phonon_wave: bool = False  # phonons as the damped linear waves of Sec. 3.4
    extra: dict = field(default_factory=dict)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def draw_couplings(seed: int = 0):
    """Four couplings log-uniform in [1e-3, 1e-1] from numpy's default_rng(seed),
    in the order (g_we, g_wp, g_ep, g_pc); g_ec = 0."""
    rng = np.random.default_rng(seed)
    g_we, g_wp, g_ep, g_pc = 10 ** rng.uniform(-3, -1, 4)
    return (float(g_we), float(g_wp), float(g_ep), 0.0, float(g_pc))


# D2Q9 FP64 slab: periodic nx = 64, 32 fluid rows, 4 solid rows per wall.
SLAB_D2Q9_FP64 = Workload(
    name="d2q9_fp64_slab_64x40", kind=9, geom="slab", nx=64, ny=40, nz=1, width=32, shell=4,
    tau=(0.8, 0.6, 1.0), G=(1e-6, 0.0, 0.0), couplings=(0.05, 0.02, 0.1, 0.0, 0.01),
    storage="fp64", steps=10_000)

# D3Q19 FP32 nanotube: 512 x 128 x 128 box, staircase pipe of radius 48 with a
# 6-cell shell, couplings drawn from seed 0.
PIPE_D3Q19_FP32 = Workload(
    name="d3q19_fp32_pipe_512x128x128_r48", kind=19, geom="pipe", nx=512, ny=128, nz=128,
    radius=48, shell=6, tau=(0.7, 0.6, 1.0), G=(1e-6, 0.0, 0.0), couplings=draw_couplings(0),
    storage="fp32", steps=5_000)

# Same nanotube scaled by 1.5 (radius 72, shell 9) and its 128 x 64 x 64
# subcase (radius 24, shell 3).
PIPE_D3Q19_LARGE = PIPE_D3Q19_FP32.with_(
    name="d3q19_pipe_768x192x192_r72", nx=768, ny=192, nz=192, radius=72, shell=9)
PIPE_D3Q19_SUB = PIPE_D3Q19_FP32.with_(
    name="d3q19_pipe_128x64x64_r24", nx=128, ny=64, nz=64, radius=24, shell=3)

# The scaled nanotube with populations stored in 16 bits (FP32 arithmetic).
PIPE_D3Q19_FP16 = PIPE_D3Q19_LARGE.with_(name="d3q19_fp16_pipe_768x192x192_r72", storage="fp16")
PIPE_D3Q19_BF16 = PIPE_D3Q19_LARGE.with_(name="d3q19_bf16_pipe_768x192x192_r72", storage="bf16")

PRESETS = {w.name: w for w in (SLAB_D2Q9_FP64, PIPE_D3Q19_FP32, PIPE_D3Q19_LARGE,
                               PIPE_D3Q19_SUB, PIPE_D3Q19_FP16, PIPE_D3Q19_BF16)}


def perturbation(w: Workload, seed: int, eps: float):
    """Random numbers of a perturbed start: drho = rho0 * eps * xi and
    u = eps * eta with xi, eta ~ U(-1, 1) from default_rng(seed), one draw
    per species, component and cell, in box order (x fastest).  u_z = 0 on
    D2Q9.  Shapes (3, nz, ny, nx) and (3, 3, nz, ny, nx)."""
    rng = np.random.default_rng(seed)
    xi = rng.uniform(-1.0, 1.0, (3, w.nz, w.ny, w.nx))
    eta = rng.uniform(-1.0, 1.0, (3, 3, w.nz, w.ny, w.nx))
    if w.kind == 9:
        eta[:, 2] = 0.0
    return w.rho0 * eps * xi, eps * eta


def channel_sweep(n: int = 96, seed: int = 0, storage: str = "fp32", scale: float = 1.0):
    """A design sweep of n independent D3Q19 channels: slab or pipe with
    probability 1/2; nx uniform in [64, 512], box cross-section ny, nz uniform
    in [16, 128] (shell included), shell uniform in [2, 8]; tau_w uniform in
    [0.55, 1.2] (tau_e 0.6, tau_p 1.0); drive g log-uniform in [1e-7, 1e-5];
    the couplings g_we, g_wp, g_ep, g_pc log-uniform in [1e-4, 1e-1],
    g_ec = 0 (a fluid cell of these channels has at most two solid faces, so
    the face-summed interface friction stays below 0.4 rho0, inside the
    stability bound).
    Draws from default_rng(seed) in that order, channel by channel.  A pipe's
    radius is the largest that fits its shell in the box (at least 2); a
    slab's fluid width is ny - 2 shell.  ``scale`` shrinks every length (for
    quick tests)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        kind = "pipe" if rng.uniform() < 0.5 else "slab"
        nx = int(rng.integers(64, 513))
        ny = int(rng.integers(16, 129))
        nz = int(rng.integers(16, 129))
        shell = int(rng.integers(2, 9))
        tau_w = float(rng.uniform(0.55, 1.2))
        g = float(10 ** rng.uniform(-7, -5))
        g_we, g_wp, g_ep, g_pc = (float(v) for v in 10 ** rng.uniform(-4, -1, 4))
        if scale != 1.0:
            nx, ny, nz = (max(8, int(round(v * scale))) for v in (nx, ny, nz))
            shell = max(1, int(round(shell * scale)))
        common = dict(name=f"sweep{seed}_{k}_{kind}", kind=19, nx=nx, ny=ny, nz=nz, shell=shell,
                      tau=(tau_w, 0.6, 1.0), G=(g, 0.0, 0.0),
                      couplings=(g_we, g_wp, g_ep, 0.0, g_pc), storage=storage)
        if kind == "pipe":
            radius = max(2, min(ny, nz) // 2 - shell)
            ny = nz = max(ny, nz, 2 * (radius + shell))
            common.update(ny=ny, nz=nz)
            out.append(Workload(geom="pipe", radius=radius, **common))
        else:
            ny = max(ny, 2 * shell + 2)
            common.update(ny=ny)
            out.append(Workload(geom="slab", width=ny - 2 * shell, **common))
    return out


@dataclass(frozen=True)
class Request:
    """One design-sweep solve of a request stream: its arrival time (s after
    the stream starts) and its channel."""
    rid: int
    arrival: float
    w: Workload


def request_stream(n: int, rate: float = 50.0, seed: int = 0, storage: str = "fp32",
                   max_cells: int = 512 * 128 * 128, min_cells: int = 32 ** 3):
    """n requests of a Poisson stream with ``rate`` arrivals per second.  Per
    request, from default_rng(seed) in this order: the inter-arrival time
    (exponential, mean 1/rate); the cell count C log-uniform in
    [min_cells, max_cells]; the aspect a uniform in [1, 4], giving
    ny = nz = round((C/a)^(1/3)) and nx = round(C/ny^2); slab or pipe with
    probability 1/2; then shell, tau_w, drive and couplings drawn as in
    channel_sweep.  The cross-section is at least 2 shell + 4 cells wide."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n):
        t += float(rng.exponential(1.0 / rate))
        c = float(np.exp(rng.uniform(np.log(min_cells), np.log(max_cells))))
        a = float(rng.uniform(1.0, 4.0))
        kind = "pipe" if rng.uniform() < 0.5 else "slab"
        shell = int(rng.integers(2, 9))
        tau_w = float(rng.uniform(0.55, 1.2))
        g = float(10 ** rng.uniform(-7, -5))
        g_we, g_wp, g_ep, g_pc = (float(v) for v in 10 ** rng.uniform(-4, -1, 4))
        ny = max(int(round((c / a) ** (1.0 / 3.0))), 2 * shell + 4)
        nx = max(1, int(round(c / ny ** 2)))
        common = dict(name=f"req{seed}_{k}_{kind}", kind=19, nx=nx, ny=ny, nz=ny, shell=shell,
                      tau=(tau_w, 0.6, 1.0), G=(g, 0.0, 0.0),
                      couplings=(g_we, g_wp, g_ep, 0.0, g_pc), storage=storage)
        if kind == "pipe":
            w = Workload(geom="pipe", radius=ny // 2 - shell, **common)
        else:
            w = Workload(geom="slab", width=ny - 2 * shell, **common)
        out.append(Request(k, t, w))
    return out


def design_grid(radii, g_we_values, nx: int = 8, shell: int = 3, tau_w: float = 0.8, G: float = 1e-6,
                g_wp: float = 0.05, g_ep: float = 0.1, g_pc: float = 0.01, storage: str = "fp32"):
    """Pipes of the given radii (box 2 (R + shell) + 2 square, nx x planes,
    x-invariant) for each water-electron coupling g_we (negative values: the
    negative quantum friction of Sec. 2): the shape of the nanotube
    permeability study of Sec. 5.1.  Other couplings fixed; g_ec = 0.  A
    steady state needs net wall friction, g_we + g_wp > 0 (with
    g_we + g_wp = 0 the water accelerates freely)."""
    out = []
    for R in radii:
        for g in g_we_values:
            n = 2 * (R + shell) + 2
            out.append(Workload(name=f"map_R{R}_g{g:+.3f}", kind=19, geom="pipe", nx=nx, ny=n, nz=n,
                                radius=R, shell=shell, tau=(tau_w, 0.6, 1.0), G=(G, 0.0, 0.0),
                                couplings=(float(g), g_wp, g_ep, 0.0, g_pc), storage=storage))
    return out
