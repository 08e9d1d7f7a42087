"""Thin Python binding of the KLB C ABI (``include/klb.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library ``_build/libklb.so``.  PyTorch provides the device buffer and the
stream.  Functions keep the C names; ``Lattice`` bundles a handle with the
torch buffer it lives in.

There is no CPU fallback: if the library cannot be loaded, or no CUDA device
is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

KLB_D2Q9, KLB_D3Q19 = 9, 19
KLB_STATIC_MAX_BLOCKS = 49152
KLB_GEOM_SLAB, KLB_GEOM_PIPE, KLB_GEOM_MASK = 0, 1, 2
KLB_FP64, KLB_FP32, KLB_FP16_DEV, KLB_BF16_DEV = 0, 1, 2, 3
STORAGE = {"fp64": KLB_FP64, "fp32": KLB_FP32, "fp16": KLB_FP16_DEV, "bf16": KLB_BF16_DEV}
KLB_IFACE_SPECULAR, KLB_IFACE_BOUNCEBACK = 0, 1
KLB_PHONON_FLUID, KLB_PHONON_WAVE = 0, 1
STATUS = {0: "KLB_OK", 1: "KLB_EINVAL", 2: "KLB_ENOMEM", 3: "KLB_ECUDA", 4: "KLB_EUNSTABLE",
          5: "KLB_ETIMEOUT", 6: "KLB_ESTATE", 7: "KLB_ERANGE"}
EXPORTS = ["klb_lattice_bytes", "klb_lattice_info", "klb_create_lattice", "klb_set_couplings",
           "klb_set_fluctuations", "klb_bounds_status", "klb_bounds_checked", "klb_init_equilibrium", "klb_step", "klb_observables", "klb_observables_static",
           "klb_get_field",
           "klb_get_state", "klb_set_state", "klb_get_step", "klb_species_cells",
           "klb_destroy", "klb_last_error", "klb_batch_bytes", "klb_batch_create",
           "klb_batch_step", "klb_batch_autotune", "klb_batch_width", "klb_batch_blocks",
           "klb_batch_destroy", "klb_batch_last_error", "klb_server_table_bytes",
           "klb_server_create", "klb_server_submit", "klb_server_tick", "klb_server_poll",
           "klb_server_get_stats", "klb_server_clock", "klb_server_destroy",
           "klb_server_last_error"]


class klb_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("geom", ctypes.c_int32), ("width", ctypes.c_int32),
                ("radius", ctypes.c_int32), ("shell", ctypes.c_int32),
                ("periodic_y", ctypes.c_int32), ("periodic_z", ctypes.c_int32),
                ("mask", ctypes.c_void_p),
                ("tau_w", ctypes.c_double), ("tau_e", ctypes.c_double),
                ("tau_p", ctypes.c_double), ("rho0", ctypes.c_double),
                ("G", ctypes.c_double * 3), ("storage", ctypes.c_int32),
                ("iface_bc", ctypes.c_int32), ("phonon_eq", ctypes.c_int32)]


class klb_couplings(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("g_we", "g_wp", "g_ep", "g_ec", "g_pc")]


class klb_obs(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("flow_rate", ctypes.c_double),
                ("fit_A", ctypes.c_double), ("fit_B", ctypes.c_double),
                ("d_wall", ctypes.c_double), ("u_slip", ctypes.c_double),
                ("dudn_wall", ctypes.c_double), ("slip_length", ctypes.c_double),
                ("u_wallrow_mean", ctypes.c_double), ("mean_u", ctypes.c_double * 3),
                ("momentum", ctypes.c_double * 3), ("mass", ctypes.c_double * 3),
                ("residual", ctypes.c_double), ("nonfinite", ctypes.c_int64),
                ("clipped", ctypes.c_int64)]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out


class klb_info(ctypes.Structure):
    _fields_ = [("fluid_cs", ctypes.c_int64), ("solid_cs", ctypes.c_int64),
                ("species_cells", ctypes.c_int64 * 3), ("active_sites", ctypes.c_int64),
                ("iface_cs", ctypes.c_int64 * 2), ("max_faces", ctypes.c_int32 * 2),
                ("d_wall", ctypes.c_double), ("bytes", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return klb_obs.as_dict(self)


class klb_server_opts(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("max_resident", ctypes.c_int32),
                ("autotune_steps", ctypes.c_int32), ("pad", ctypes.c_int32)]


class klb_request(ctypes.Structure):
    _fields_ = [("desc", klb_desc), ("couplings", klb_couplings), ("tol", ctypes.c_double),
                ("max_steps", ctypes.c_int64), ("max_seconds", ctypes.c_double),
                ("arrival", ctypes.c_double), ("id", ctypes.c_int64)]


class klb_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("steps", ctypes.c_int64), ("sites", ctypes.c_int64), ("bytes", ctypes.c_uint64),
                ("arrival", ctypes.c_double), ("admitted", ctypes.c_double),
                ("finished", ctypes.c_double), ("obs", klb_obs)]

    def as_dict(self) -> dict:
        out = {n: getattr(self, n) for n, _ in self._fields_ if n not in ("pad", "obs")}
        out["obs"] = self.obs.as_dict()
        return out


class klb_server_stats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int64), ("resident", ctypes.c_int64),
                ("finished", ctypes.c_int64), ("rounds", ctypes.c_int64),
                ("batch_forms", ctypes.c_int64), ("arena_bytes", ctypes.c_uint64),
                ("bytes_in_use", ctypes.c_uint64), ("peak_bytes_in_use", ctypes.c_uint64),
                ("table_bytes", ctypes.c_uint64), ("site_updates", ctypes.c_double),
                ("width", ctypes.c_int32), ("pad", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_ if n != "pad"}


class KLBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str | None = None):
    """Load libklb.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(path or os.environ.get("KLB_LIBRARY") or _build.build())
    P, I32, I64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    lib.klb_lattice_bytes.restype = SZ
    lib.klb_lattice_bytes.argtypes = [ctypes.POINTER(klb_desc)]
    lib.klb_lattice_info.restype = I32
    lib.klb_lattice_info.argtypes = [ctypes.POINTER(klb_desc), ctypes.POINTER(klb_info)]
    lib.klb_create_lattice.restype = I32
    lib.klb_create_lattice.argtypes = [ctypes.POINTER(klb_desc), P, SZ, P, ctypes.POINTER(P)]
    lib.klb_set_couplings.restype = I32
    lib.klb_set_couplings.argtypes = [P, ctypes.POINTER(klb_couplings)]
    lib.klb_bounds_status.restype = I32
    lib.klb_bounds_status.argtypes = [P, ctypes.POINTER(ctypes.c_uint32)]
    lib.klb_bounds_checked.restype = ctypes.c_int
    lib.klb_bounds_checked.argtypes = []
    lib.klb_set_fluctuations.restype = I32
    lib.klb_set_fluctuations.argtypes = [P, ctypes.c_double, ctypes.c_uint64]
    lib.klb_init_equilibrium.restype = I32
    lib.klb_init_equilibrium.argtypes = [P, P, P]
    lib.klb_step.restype = I32
    lib.klb_step.argtypes = [P, I64]
    lib.klb_observables.restype = I32
    lib.klb_observables.argtypes = [P, ctypes.POINTER(klb_obs)]
    lib.klb_observables_static.restype = I32
    lib.klb_observables_static.argtypes = [P, ctypes.POINTER(klb_obs)]
    lib.klb_get_field.restype = I32
    lib.klb_get_field.argtypes = [P, P, P]
    lib.klb_get_state.restype = I32
    lib.klb_get_state.argtypes = [P, P, P, P]
    lib.klb_set_state.restype = I32
    lib.klb_set_state.argtypes = [P, P, P, P, I64]
    lib.klb_get_step.restype = I64
    lib.klb_get_step.argtypes = [P]
    lib.klb_species_cells.restype = I64
    lib.klb_species_cells.argtypes = [P, I32]
    lib.klb_destroy.restype = I32
    lib.klb_destroy.argtypes = [P]
    lib.klb_last_error.restype = ctypes.c_char_p
    lib.klb_last_error.argtypes = [P]
    lib.klb_batch_bytes.restype = SZ
    lib.klb_batch_bytes.argtypes = [ctypes.POINTER(P), ctypes.c_int]
    lib.klb_batch_create.restype = I32
    lib.klb_batch_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, P, SZ, ctypes.POINTER(P)]
    lib.klb_batch_step.restype = I32
    lib.klb_batch_step.argtypes = [P, I64]
    lib.klb_batch_autotune.restype = I32
    lib.klb_batch_autotune.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.klb_batch_width.restype = ctypes.c_int
    lib.klb_batch_width.argtypes = [P]
    lib.klb_batch_blocks.restype = I64
    lib.klb_batch_blocks.argtypes = [P]
    lib.klb_batch_destroy.restype = I32
    lib.klb_batch_destroy.argtypes = [P]
    lib.klb_batch_last_error.restype = ctypes.c_char_p
    lib.klb_batch_last_error.argtypes = [P]
    lib.klb_server_table_bytes.restype = SZ
    lib.klb_server_table_bytes.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.klb_server_create.restype = I32
    lib.klb_server_create.argtypes = [P, SZ, P, ctypes.POINTER(klb_server_opts), ctypes.POINTER(P)]
    lib.klb_server_submit.restype = I32
    lib.klb_server_submit.argtypes = [P, ctypes.POINTER(klb_request)]
    lib.klb_server_tick.restype = I32
    lib.klb_server_tick.argtypes = [P, ctypes.POINTER(I64)]
    lib.klb_server_poll.restype = I64
    lib.klb_server_poll.argtypes = [P, ctypes.POINTER(klb_result), I64]
    lib.klb_server_get_stats.restype = I32
    lib.klb_server_get_stats.argtypes = [P, ctypes.POINTER(klb_server_stats)]
    lib.klb_server_clock.restype = ctypes.c_double
    lib.klb_server_clock.argtypes = [P]
    lib.klb_server_destroy.restype = I32
    lib.klb_server_destroy.argtypes = [P]
    lib.klb_server_last_error.restype = ctypes.c_char_p
    lib.klb_server_last_error.argtypes = [P]
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(st, handle=None):
    if st != 0:
        msg = _lib.klb_last_error(handle).decode(errors="replace")
        raise KLBError(st, msg)


def make_desc(kind=KLB_D3Q19, nx=1, ny=1, nz=1, geom=KLB_GEOM_PIPE, width=0, radius=0, shell=0,
              mask=None, periodic_y=False, periodic_z=False, tau=(0.8, 0.6, 1.0), rho0=1.0,
              G=(0.0, 0.0, 0.0), storage=KLB_FP32, iface_bc=KLB_IFACE_SPECULAR,
              phonon_eq=0):
    """Fill a klb_desc.  ``mask`` (MASK geometry) is a (nz, ny) uint8 array;
    the returned object keeps a reference to it."""
    d = klb_desc()
    d.kind, d.nx, d.ny, d.nz, d.geom = kind, nx, ny, nz, geom
    d.width, d.radius, d.shell = width, radius, shell
    d.periodic_y, d.periodic_z = int(bool(periodic_y)), int(bool(periodic_z))
    d._mask_keep = None
    if mask is not None:
        m = np.ascontiguousarray(np.asarray(mask, np.uint8).reshape(nz, ny))
        d._mask_keep = m
        d.mask = m.ctypes.data
    d.tau_w, d.tau_e, d.tau_p = tau
    d.rho0 = rho0
    d.G[0], d.G[1], d.G[2] = G
    d.storage, d.iface_bc = storage, iface_bc
    d.phonon_eq = phonon_eq
    return d


def klb_lattice_bytes(desc: klb_desc) -> int:
    return int(load_library().klb_lattice_bytes(ctypes.byref(desc)))


def klb_lattice_info(desc: klb_desc) -> dict:
    lib = load_library()
    info = klb_info()
    _check(lib.klb_lattice_info(ctypes.byref(desc), ctypes.byref(info)))
    return info.as_dict()


class Lattice:
    """A lattice living in a torch-allocated device buffer on the current
    CUDA stream of ``device``."""

    def __init__(self, desc: klb_desc, device="cuda", stream=None):
        import torch

        lib = load_library()
        if not torch.cuda.is_available():
            raise KLBError(3, "no CUDA device: the KLB library has no CPU path")
        self.desc = desc
        self.nbytes = klb_lattice_bytes(desc)
        if self.nbytes == 0:
            h = ctypes.c_void_p()
            _check(lib.klb_create_lattice(ctypes.byref(desc), None, 0, None, ctypes.byref(h)))
        self.device = torch.device(device)
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib.klb_create_lattice(ctypes.byref(desc), ctypes.c_void_p(self.buf.data_ptr()),
                                          self.nbytes, ctypes.c_void_p(self.stream.cuda_stream),
                                          ctypes.byref(self._h)))
        self.ncell = desc.nx * desc.ny * desc.nz
        self.Q = desc.kind

    # -- C entry points -------------------------------------------------
    def set_couplings(self, g_we, g_wp, g_ep, g_ec=0.0, g_pc=0.0):
        c = klb_couplings(g_we, g_wp, g_ep, g_ec, g_pc)
        _check(_lib.klb_set_couplings(self._h, ctypes.byref(c)), self._h)

    def bounds_status(self) -> int:
        """First out-of-range index site recorded by a debug build (0: none);
        clears it."""
        v = ctypes.c_uint32()
        _check(_lib.klb_bounds_status(self._h, ctypes.byref(v)), self._h)
        return v.value

    def set_fluctuations(self, kT: float, seed: int = 0):
        """Thermal noise of the water populations (klb_set_fluctuations)."""
        _check(_lib.klb_set_fluctuations(self._h, float(kT), int(seed)), self._h)

    def init_equilibrium(self, drho=None, u=None):
        d = None if drho is None else np.ascontiguousarray(drho, np.float64)
        v = None if u is None else np.ascontiguousarray(u, np.float64)
        if d is not None:
            assert d.size == 3 * self.ncell
        if v is not None:
            assert v.size == 9 * self.ncell
        _check(_lib.klb_init_equilibrium(self._h, _ptr(d), _ptr(v)), self._h)

    def step(self, n: int = 1):
        _check(_lib.klb_step(self._h, int(n)), self._h)

    def observables(self, allow_unstable=False) -> dict:
        o = klb_obs()
        st = _lib.klb_observables(self._h, ctypes.byref(o))
        if not (allow_unstable and st in (4, 7)):
            _check(st, self._h)
        return o.as_dict()

    def _box(self, *lead):
        return (*lead, self.desc.nz, self.desc.ny, self.desc.nx)

    def get_field(self):
        drho = np.zeros(self._box(3))
        u = np.zeros(self._box(3, 3))
        _check(_lib.klb_get_field(self._h, _ptr(drho), _ptr(u)), self._h)
        return drho, u

    def get_state(self):
        g = np.zeros(self._box(3, self.Q))
        U1 = np.zeros(self._box(3, 3))
        U2 = np.zeros(self._box(3, 3))
        _check(_lib.klb_get_state(self._h, _ptr(g), _ptr(U1), _ptr(U2)), self._h)
        return g, U1, U2

    def set_state(self, g, U1, U2, step=0):
        g = np.ascontiguousarray(g, np.float64)
        U1 = np.ascontiguousarray(U1, np.float64)
        U2 = np.ascontiguousarray(U2, np.float64)
        _check(_lib.klb_set_state(self._h, _ptr(g), _ptr(U1), _ptr(U2), int(step)), self._h)

    @property
    def nstep(self) -> int:
        return int(_lib.klb_get_step(self._h))

    def species_cells(self, s: int) -> int:
        return int(_lib.klb_species_cells(self._h, s))

    def active_sites(self) -> int:
        """Fluid + solid cells (each solid cell carries electrons and phonons)."""
        return self.species_cells(0) + self.species_cells(1)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(_lib.klb_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many lattices stepped together, one launch per step (klb_batch_*).
    The members must share kind, storage, stream and time level."""

    def __init__(self, members):
        import torch

        lib = load_library()
        self.members = list(members)
        arr = (ctypes.c_void_p * len(self.members))(*[m._h.value for m in self.members])
        self._arr = arr
        n = lib.klb_batch_bytes(arr, len(self.members))
        if n == 0:
            raise KLBError(1, "these lattices cannot form a batch")
        self.buf = torch.empty(n, dtype=torch.uint8, device=self.members[0].device)
        self._h = ctypes.c_void_p()
        st = lib.klb_batch_create(arr, len(self.members), ctypes.c_void_p(self.buf.data_ptr()), n,
                                  ctypes.byref(self._h))
        _check(st)

    def _bcheck(self, st):
        if st != 0:
            raise KLBError(st, _lib.klb_batch_last_error(self._h).decode(errors="replace"))

    def step(self, n: int = 1):
        self._bcheck(_lib.klb_batch_step(self._h, int(n)))

    def autotune(self, steps_per_candidate: int = 5) -> int:
        w = ctypes.c_int()
        self._bcheck(_lib.klb_batch_autotune(self._h, int(steps_per_candidate), ctypes.byref(w)))
        return w.value

    @property
    def width(self) -> int:
        return int(_lib.klb_batch_width(self._h))

    @property
    def blocks(self) -> int:
        return int(_lib.klb_batch_blocks(self._h))

    def active_sites(self) -> int:
        return sum(m.active_sites() for m in self.members)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.klb_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def klb_server_table_bytes(storage: int, max_resident: int) -> int:
    return int(load_library().klb_server_table_bytes(storage, max_resident))


class Server:
    """Request loop over a torch-allocated device arena of ``arena_bytes``
    (klb_server_*): submit requests at any time, call ``tick`` to run one
    scheduling round, ``poll`` for finished results."""

    def __init__(self, arena_bytes: int, kind=KLB_D3Q19, storage="fp32", check_every=64,
                 max_resident=128, autotune_steps=0, device="cuda", stream=None):
        import torch

        lib = load_library()
        if not torch.cuda.is_available():
            raise KLBError(3, "no CUDA device: the KLB library has no CPU path")
        self.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        self.kind = int(kind)
        self.device = torch.device(device)
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        o = klb_server_opts(self.kind, self.storage, int(check_every), int(max_resident),
                            int(autotune_steps), 0)
        self._h = ctypes.c_void_p()
        st = lib.klb_server_create(ctypes.c_void_p(self.arena.data_ptr()), int(arena_bytes),
                                   ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(o),
                                   ctypes.byref(self._h))
        if st != 0:
            raise KLBError(st, lib.klb_server_last_error(None).decode(errors="replace"))
        self._keep = {}

    def _scheck(self, st):
        if st != 0:
            raise KLBError(st, _lib.klb_server_last_error(self._h).decode(errors="replace"))

    def submit(self, desc: klb_desc, couplings, tol: float, max_steps: int, req_id: int,
               arrival: float = -1.0, max_seconds: float = 0.0):
        r = klb_request(desc, klb_couplings(*couplings), float(tol), int(max_steps),
                        float(max_seconds), float(arrival), int(req_id))
        self._scheck(_lib.klb_server_submit(self._h, ctypes.byref(r)))

    def tick(self) -> int:
        n = ctypes.c_int64()
        self._scheck(_lib.klb_server_tick(self._h, ctypes.byref(n)))
        return n.value

    def poll(self, max_results: int = 1024) -> list:
        out = (klb_result * max_results)()
        n = _lib.klb_server_poll(self._h, out, max_results)
        return [out[k].as_dict() for k in range(n)]

    def stats(self) -> dict:
        st = klb_server_stats()
        self._scheck(_lib.klb_server_get_stats(self._h, ctypes.byref(st)))
        return st.as_dict()

    def clock(self) -> float:
        return float(_lib.klb_server_clock(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.klb_server_destroy(self._h)
            self._h = ctypes.c_void_p()
        self.arena = None  # the caller-side buffer goes back to torch's allocator

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def residual_is_valid(obs: dict) -> bool:
    return not math.isnan(obs["residual"])


def desc_from_workload(w, nx=None) -> klb_desc:
    """klb_desc of an ``inputs.Workload`` (optionally with another nx)."""
    geom = {"slab": KLB_GEOM_SLAB, "pipe": KLB_GEOM_PIPE, "mask": KLB_GEOM_MASK}[w.geom]
    storage = STORAGE[w.storage]
    iface = {"specular": KLB_IFACE_SPECULAR, "bounceback": KLB_IFACE_BOUNCEBACK}[w.iface_bc]
    return make_desc(kind=w.kind, nx=nx or w.nx, ny=w.ny, nz=w.nz, geom=geom, width=w.width,
                     radius=w.radius, shell=w.shell, mask=w.extra.get("mask"),
                     periodic_y=w.extra.get("periodic_y", False),
                     periodic_z=w.extra.get("periodic_z", False), tau=w.tau, rho0=w.rho0,
                     G=w.G, storage=storage, iface_bc=iface,
                     phonon_eq=KLB_PHONON_WAVE if w.phonon_wave else KLB_PHONON_FLUID)


def lattice_from_workload(w, device="cuda", stream=None) -> Lattice:
    lat = Lattice(desc_from_workload(w), device=device, stream=stream)
    lat.set_couplings(*w.couplings)
    return lat
