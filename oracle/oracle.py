"""Python side of the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

The time step itself is the plain C code in ``klb_oracle.c`` (loaded with
ctypes).  This module adds, in plain numpy:

* the geometry of the paper's set-ups (Sec. 2: a nanochannel, slab or
  cylindrical nanotube, with solid walls), as a cross-section type map;
* the observables, written out from their definitions: flow rate, the slip
  length L_s = u_s / (du/dn)_w of Sec. 1, the wall-row mean velocity, species
  masses, momenta and mean velocities, and the steady-state residual;
* the slip-Poiseuille closed forms used to pin the oracle (Sec. 1: slip turns
  the D^-4 pressure scaling into D^-2).

Parity status.  Pinned (tests/test_oracle_pins.py): lattice tables and the
moment identities of the equilibrium and the Guo source; the streaming /
boundary rule (bijectivity, specular reflection, bounce-back); mass and
momentum balance per step; closed-form special cases (free acceleration,
Crank-Nicolson e-p relaxation, lagged water-electron pair); the magic-tau
bounce-back parabola; bulk curvature; wall force balance; an independent
dense steady-state solve of the slab; slip-Poiseuille closed forms; D3Q19
slab = D2Q9 slab; eight-fold pipe symmetry; the phonon damped-wave variant
of Sec. 3.4 (moments of its linear equilibrium, the decay rate and frequency
of a single Fourier mode of the damped wave equation, no advection by a
uniform phonon flow).  Parity unpinned: the
Bose-Einstein / Fermi-Dirac specific corrections to the equilibria, which the
paper does not give and which are therefore not implemented.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "klb_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libklb_oracle.so")

T_VOID, T_FLUID, T_SOLID = 0, 1, 2
WATER, ELECTRON, PHONON = 0, 1, 2
K0_FIT = 4  # fit excludes fluid cells closer than this to the interface


def build_oracle(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/_build`` (plain gcc, no GPU)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    os.makedirs(_LIB_DIR, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O3", "-std=c99", "-fPIC", "-shared", _SRC,
                           "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build_oracle())
    P, D, I, L = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_long
    lib.kor_create.restype = P
    lib.kor_create.argtypes = [I, I, I, I, I, I, P]
    lib.kor_destroy.argtypes = [P]
    lib.kor_set_params.argtypes = [P, D, D, D, D, D, D, D, I]
    lib.kor_set_couplings.argtypes = [P, D, D, D, D, D]
    lib.kor_set_fluctuations.argtypes = [P, D, ctypes.c_uint64]
    lib.kor_philox.argtypes = [P, P, P]
    lib.kor_init_equilibrium.argtypes = [P, P, P]
    lib.kor_step.argtypes = [P, L]
    lib.kor_observe.argtypes = [P, P, P, P, P]
    lib.kor_get_step.restype = L
    lib.kor_get_step.argtypes = [P]
    lib.kor_get_state.argtypes = [P, P, P, P]
    lib.kor_set_state.argtypes = [P, P, P, P, L]
    lib.kor_stream_table.argtypes = [P, I, P, P]
    lib.kor_lattice.argtypes = [P, P, P, P]
    lib.kor_geq.restype = D
    lib.kor_geq.argtypes = [P, I, D, D, D, D]
    lib.kor_guo.restype = D
    lib.kor_guo.argtypes = [P, I, D, D, D, D, D, D, D]
    lib.kor_geq_species.restype = D
    lib.kor_geq_species.argtypes = [P, I, I, D, D, D, D]
    lib.kor_guo_species.restype = D
    lib.kor_guo_species.argtypes = [P, I, I, D, D, D, D, D, D, D]
    lib.kor_set_phonon_wave.argtypes = [P, I]
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# Geometry (Sec. 2 set-up: water in a nanochannel between solid walls)

@dataclass
class Geometry:
    """Cross-section of an x-invariant channel.

    ``cs_type[z, y]`` is 0 void, 1 fluid, 2 solid.  ``dist[z, y]`` is the
    distance of a cell centre (y+1/2, z+1/2) from the channel centre plane
    (slab) or axis (pipe); ``d_wall`` the wall position used by the slip fit:
    the half width h for a slab, R_eff = sqrt(fluid cells per slice / pi) for a
    staircase pipe.
    """
    cs_type: np.ndarray
    periodic_y: bool
    periodic_z: bool
    dist: np.ndarray | None
    d_wall: float
    kind: str

    @property
    def ny(self):
        return self.cs_type.shape[1]

    @property
    def nz(self):
        return self.cs_type.shape[0]


def cross_section(geom: str, ny: int, nz: int, width: int = 0, radius: int = 0,
                  shell: int = 0, mask=None, periodic_y=False,
                  periodic_z=False) -> Geometry:
    """Build the cross-section type map.

    slab: ``width`` fluid rows centred in y, ``shell`` solid rows on each
      side, void beyond; walls normal to y; periodic in z.
    pipe: axis at (ny/2, nz/2); fluid where r < R, solid where
      R <= r < R + shell, void elsewhere (r of the cell centre, compared
      exactly in doubled integer coordinates).
    mask: the given map (shape (nz, ny)), with the given periodicity.
    """
    if geom == "slab":
        t = np.zeros((nz, ny), np.uint8)
        y0 = (ny - width) // 2
        for y in range(ny):
            if y0 <= y < y0 + width:
                t[:, y] = T_FLUID
            elif y0 - shell <= y < y0 + width + shell:
                t[:, y] = T_SOLID
        yc = y0 + width / 2.0
        dist = np.abs(np.arange(ny) + 0.5 - yc)[None, :].repeat(nz, 0)
        return Geometry(t, False, True, dist, width / 2.0, "slab")
    if geom == "pipe":
        y = np.arange(ny)[None, :]
        z = np.arange(nz)[:, None]
        r2x4 = (2 * y + 1 - ny) ** 2 + (2 * z + 1 - nz) ** 2
        t = np.zeros((nz, ny), np.uint8)
        t[r2x4 < (2 * (radius + shell)) ** 2] = T_SOLID
        t[r2x4 < (2 * radius) ** 2] = T_FLUID
        dist = np.sqrt(r2x4) / 2.0
        r_eff = float(np.sqrt((t == T_FLUID).sum() / np.pi))
        return Geometry(t, False, False, dist, r_eff, "pipe")
    if geom == "mask":
        t = np.ascontiguousarray(np.asarray(mask, np.uint8).reshape(nz, ny))
        return Geometry(t, bool(periodic_y), bool(periodic_z), None, float("nan"), "mask")
    raise ValueError(geom)


# --------------------------------------------------------------------------

class Oracle:
    """One lattice of the three-species scheme, FP64, on the CPU."""

    def __init__(self, Q: int, nx: int, geo: Geometry, tau=(0.8, 0.6, 1.0), rho0=1.0,
                 G=(0.0, 0.0, 0.0), couplings=(0.0, 0.0, 0.0, 0.0, 0.0),
                 iface_bounceback=False, phonon_wave=False):
        lib = _load()
        self.Q, self.nx, self.geo = Q, nx, geo
        self.ny, self.nz = geo.ny, geo.nz
        self.ncell = nx * self.ny * self.nz
        self.rho0 = rho0
        self.tau = tuple(tau)
        self.G = tuple(G)
        cs = np.ascontiguousarray(geo.cs_type.astype(np.uint8))
        h = lib.kor_create(Q, nx, self.ny, self.nz, int(geo.periodic_y),
                           int(geo.periodic_z), _ptr(cs))
        if not h:
            raise ValueError("oracle: bad lattice shape")
        self._h = ctypes.c_void_p(h)
        lib.kor_set_params(self._h, tau[0], tau[1], tau[2], rho0, G[0], G[1], G[2],
                           int(bool(iface_bounceback)))
        lib.kor_set_phonon_wave(self._h, int(bool(phonon_wave)))
        self.phonon_wave = bool(phonon_wave)
        self.set_couplings(*couplings)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.kor_destroy(h)
            self._h = None

    # shapes
    def _box(self, *lead):
        return (*lead, self.nz, self.ny, self.nx)

    def set_fluctuations(self, kT: float, seed: int):
        """Thermal noise of the water populations (0 disables)."""
        _lib.kor_set_fluctuations(self._h, float(kT), int(seed))

    def set_couplings(self, g_we, g_wp, g_ep, g_ec=0.0, g_pc=0.0):
        self.couplings = (g_we, g_wp, g_ep, g_ec, g_pc)
        _lib.kor_set_couplings(self._h, g_we, g_wp, g_ep, g_ec, g_pc)

    def init_equilibrium(self, drho=None, u=None):
        """drho: (3, nz, ny, nx); u: (3, 3, nz, ny, nx); None means zero."""
        d = None if drho is None else np.ascontiguousarray(drho, np.float64).reshape(self._box(3))
        v = None if u is None else np.ascontiguousarray(u, np.float64).reshape(self._box(3, 3))
        _lib.kor_init_equilibrium(self._h, _ptr(d), _ptr(v))

    def step(self, n: int = 1):
        _lib.kor_step(self._h, int(n))

    @property
    def nstep(self) -> int:
        return int(_lib.kor_get_step(self._h))

    def observe(self):
        """Fields of the current step: drho (3,...), u (3,3,...), F (3,3,...), uprev."""
        drho = np.zeros(self._box(3))
        u = np.zeros(self._box(3, 3))
        F = np.zeros(self._box(3, 3))
        up = np.zeros(self._box(3, 3))
        _lib.kor_observe(self._h, _ptr(drho), _ptr(u), _ptr(F), _ptr(up))
        return {"drho": drho, "u": u, "F": F, "uprev": up, "step": self.nstep}

    def get_state(self):
        """(g*, U, U2): post-collision deviations (3, Q, ...) and the
        velocities of the two previous steps (3, 3, ...)."""
        gs = np.zeros(self._box(3, self.Q))
        U = np.zeros(self._box(3, 3))
        U2 = np.zeros(self._box(3, 3))
        _lib.kor_get_state(self._h, _ptr(gs), _ptr(U), _ptr(U2))
        return gs, U, U2

    def set_state(self, gs, U, U2, step=0):
        gs = np.ascontiguousarray(gs, np.float64).reshape(self._box(3, self.Q))
        U = np.ascontiguousarray(U, np.float64).reshape(self._box(3, 3))
        U2 = np.ascontiguousarray(U2, np.float64).reshape(self._box(3, 3))
        _lib.kor_set_state(self._h, _ptr(gs), _ptr(U), _ptr(U2), int(step))

    def stream_table(self, s: int):
        src = np.zeros((self.Q, self.ncell), np.int64)
        sd = np.zeros((self.Q, self.ncell), np.int32)
        _lib.kor_stream_table(self._h, s, _ptr(src), _ptr(sd))
        return src, sd

    def lattice(self):
        c = np.zeros((self.Q, 3), np.int32)
        w = np.zeros(self.Q)
        opp = np.zeros(self.Q, np.int32)
        _lib.kor_lattice(self._h, _ptr(c), _ptr(w), _ptr(opp))
        return c, w, opp

    def geq(self, i, drho, u):
        return _lib.kor_geq(self._h, i, drho, u[0], u[1], u[2])

    def guo(self, i, omega, u, F):
        return _lib.kor_guo(self._h, i, omega, u[0], u[1], u[2], F[0], F[1], F[2])

    def geq_species(self, s, i, drho, u):
        """Equilibrium of direction i for species s (the phonons' is linear
        under the damped-wave variant of Sec. 3.4)."""
        return _lib.kor_geq_species(self._h, s, i, drho, u[0], u[1], u[2])

    def guo_species(self, s, i, omega, u, F):
        return _lib.kor_guo_species(self._h, s, i, omega, u[0], u[1], u[2], F[0], F[1], F[2])

    def species_mask(self, s):
        t = T_FLUID if s == WATER else T_SOLID
        return np.broadcast_to((self.geo.cs_type == t)[:, :, None], self._box())

    def observables(self, fields=None):
        f = self.observe() if fields is None else fields
        return observables_from_fields(self.geo, self.nx, self.rho0, f)


# --------------------------------------------------------------------------
# Observables, from their definitions

def _solid_face_count(geo: Geometry) -> np.ndarray:
    """Number of solid face-neighbours (+-y, +-z) of each cross-section cell."""
    t = geo.cs_type
    nz, ny = t.shape
    cnt = np.zeros_like(t, dtype=np.int32)
    for z in range(nz):
        for y in range(ny):
            for dy, dz in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                yy, zz = y + dy, z + dz
                if not (0 <= yy < ny):
                    if not geo.periodic_y:
                        continue
                    yy %= ny
                if not (0 <= zz < nz):
                    if not geo.periodic_z:
                        continue
                    zz %= nz
                if t[zz, yy] == T_SOLID:
                    cnt[z, y] += 1
    return cnt


def observables_from_fields(geo: Geometry, nx: int, rho0: float, f: dict) -> dict:
    """Observables of one step from dense fields (see module docstring).

    flow_rate  = (1/nx) sum over fluid cells of u_x;
    fit        = least squares u_x = A + B d^2 over fluid cells at least
                 K0_FIT from the wall (d_wall - d >= K0_FIT);
    u_slip     = A + B d_wall^2, dudn_wall = |2 B d_wall|,
    slip_length = u_slip / dudn_wall (Sec. 1);
    u_wallrow_mean = mean u_x over fluid cells with a solid face-neighbour;
    mass[s] = sum (rho_s - rho0), momentum[s] = sum rho_s u_x,s,
    mean_u[s] = mean u_x,s over the cells of s;
    residual = max over all species cells of |u_x(n) - u_x(n-1)| (NaN at n = 0).
    """
    t = geo.cs_type
    fluid = np.broadcast_to((t == T_FLUID)[:, :, None], (geo.nz, geo.ny, nx))
    solid = np.broadcast_to((t == T_SOLID)[:, :, None], (geo.nz, geo.ny, nx))
    masks = [fluid, solid, solid]
    u, drho, up = f["u"], f["drho"], f["uprev"]
    out = {"step": int(f["step"])}
    ux = u[0, 0]
    out["flow_rate"] = float(ux[fluid].sum() / nx)
    if geo.dist is not None:
        d = np.broadcast_to(geo.dist[:, :, None], (geo.nz, geo.ny, nx))
        sel = fluid & ((geo.d_wall - d) >= K0_FIT)
        Amat = np.stack([np.ones(sel.sum()), d[sel] ** 2], axis=1)
        (A, B), *_ = np.linalg.lstsq(Amat, ux[sel], rcond=None)
        out["fit_A"], out["fit_B"] = float(A), float(B)
        out["u_slip"] = float(A + B * geo.d_wall ** 2)
        out["dudn_wall"] = float(abs(2.0 * B * geo.d_wall))
        out["slip_length"] = out["u_slip"] / out["dudn_wall"] if out["dudn_wall"] else float("inf")
    else:
        for k in ("fit_A", "fit_B", "u_slip", "dudn_wall", "slip_length"):
            out[k] = float("nan")
    wall = np.broadcast_to((_solid_face_count(geo) > 0)[:, :, None], fluid.shape) & fluid
    out["u_wallrow_mean"] = float(ux[wall].mean()) if wall.any() else float("nan")
    out["mean_u"], out["momentum"], out["mass"] = [], [], []
    res = 0.0
    for s in range(3):
        m = masks[s]
        if not m.any():
            out["mean_u"].append(float("nan"))
            out["momentum"].append(0.0)
            out["mass"].append(0.0)
            continue
        out["mean_u"].append(float(u[s, 0][m].mean()))
        out["momentum"].append(float(((rho0 + drho[s]) * u[s, 0])[m].sum()))
        out["mass"].append(float(drho[s][m].sum()))
        res = max(res, float(np.abs(u[s, 0][m] - up[s, 0][m]).max()))
    out["residual"] = res if out["step"] > 0 else float("nan")
    out["nonfinite"] = int(sum((~np.isfinite(u[s][:, masks[s]])).sum() +
                               (~np.isfinite(drho[s][masks[s]])).sum() for s in range(3)))
    return out


# --------------------------------------------------------------------------
# Slip-Poiseuille closed forms (Sec. 1), lattice units, nu = (tau - 1/2) / 3

def slip_poiseuille_slab(G, rho, tau, h, Ls):
    """u(d) = G/(2 rho nu) (h^2 - d^2) + u_s ;  flow per unit depth
    Q = 2 G h^3 / (3 rho nu) (1 + 3 L_s / h)."""
    nu = (tau - 0.5) / 3.0
    us = Ls * G * h / (rho * nu)
    prof = lambda d: G / (2 * rho * nu) * (h * h - np.asarray(d) ** 2) + us  # noqa: E731
    Q = 2 * G * h ** 3 / (3 * rho * nu) * (1 + 3 * Ls / h)
    return prof, Q


def slip_poiseuille_pipe(G, rho, tau, R, Ls):
    """u(r) = G/(4 rho nu) (R^2 - r^2) + u_s ;  Q = pi G R^4 / (8 rho nu) (1 + 4 L_s / R)."""
    nu = (tau - 0.5) / 3.0
    us = Ls * G * R / (2 * rho * nu)
    prof = lambda r: G / (4 * rho * nu) * (R * R - np.asarray(r) ** 2) + us  # noqa: E731
    Q = np.pi * G * R ** 4 / (8 * rho * nu) * (1 + 4 * Ls / R)
    return prof, Q


def philox4x32_10(ctr, key):
    """The oracle's Philox-4x32-10 words for a counter (4 words) and key (2)."""
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    _load().kor_philox(c.ctypes.data_as(ctypes.c_void_p), k.ctypes.data_as(ctypes.c_void_p),
                    out.ctypes.data_as(ctypes.c_void_p))
    return out
