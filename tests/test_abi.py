"""CPU tests of the C ABI library: it builds, loads without a GPU, exports
every entry point declared in include/klb.h, and its host-side geometry
(rows, interface cells, fit wall) agrees with the oracle's independent one."""
import math
import os
import re

import numpy as np
import pytest

from klb_testutil import oracle_geometry
from oracle.oracle import _solid_face_count
from paper_2403_15768_gb300 import inputs, klb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_entry_point():
    lib = klb.load_library()
    with open(os.path.join(ROOT, "include", "klb.h")) as fh:
        header = fh.read()
    declared = set(re.findall(r"^\s*(?:klb_status|size_t|int64_t|int|double|const char \*)\s*\*?\s*(klb_\w+)\s*\(",
                              header, re.M))
    assert {"klb_create_lattice", "klb_step", "klb_observables", "klb_set_couplings"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(klb.EXPORTS)


def _geometry_cases():
    yield inputs.SLAB_D2Q9_FP64
    yield inputs.PIPE_D3Q19_FP32
    yield inputs.PIPE_D3Q19_LARGE
    yield inputs.PIPE_D3Q19_SUB
    yield inputs.PIPE_D3Q19_SUB.with_(name="odd", nx=37, ny=17, nz=15, radius=5, shell=2)
    yield inputs.PIPE_D3Q19_SUB.with_(name="thin", nx=5, ny=12, nz=12, radius=3, shell=1)
    yield inputs.SLAB_D2Q9_FP64.with_(name="slab3d", kind=19, nx=9, ny=14, nz=3, width=6, shell=3,
                                      storage="fp32")


@pytest.mark.parametrize("w", list(_geometry_cases()), ids=lambda w: w.name)
def test_host_geometry_matches_oracle(w):
    info = klb.klb_lattice_info(klb.desc_from_workload(w))
    geo = oracle_geometry(w)
    nf = int((geo.cs_type == 1).sum())
    ns = int((geo.cs_type == 2).sum())
    assert info["fluid_cs"] == nf and info["solid_cs"] == ns
    assert info["species_cells"] == [nf * w.nx, ns * w.nx, ns * w.nx]
    assert info["active_sites"] == (nf + ns) * w.nx
    faces = _solid_face_count(geo)
    assert info["iface_cs"][0] == int(((geo.cs_type == 1) & (faces > 0)).sum())
    assert info["max_faces"][0] == int(faces[geo.cs_type == 1].max())
    assert info["d_wall"] == pytest.approx(geo.d_wall, rel=0, abs=0)
    assert info["bytes"] == klb.klb_lattice_bytes(klb.desc_from_workload(w)) > 0


def test_nanotube_counts():
    """The 512x128x128 staircase nanotube of radius 48 and shell 6."""
    info = klb.klb_lattice_info(klb.desc_from_workload(inputs.PIPE_D3Q19_FP32))
    assert (info["fluid_cs"], info["solid_cs"]) == (7232, 1944)
    assert info["active_sites"] == 4_698_112
    assert sum(info["species_cells"]) == 5_693_440


@pytest.mark.parametrize("change,msg", [
    (dict(tau=(0.5, 0.6, 1.0)), "relaxation"),
    (dict(tau=(0.8, float("nan"), 1.0)), "non-finite"),
    (dict(rho0=0.0), "rho0"),
    (dict(nz=2), "D2Q9"),
    (dict(shell=0), "slab"),
    (dict(width=40), "slab"),
])
def test_invalid_descriptions_are_rejected(change, msg):
    w = inputs.SLAB_D2Q9_FP64.with_(**change)
    d = klb.desc_from_workload(w)
    assert klb.klb_lattice_bytes(d) == 0
    with pytest.raises(klb.KLBError) as e:
        klb.klb_lattice_info(d)
    assert e.value.status == 1 and msg in str(e.value)


def test_phonon_equilibrium_option_is_validated():
    """klb_desc.phonon_eq accepts the default second-order equilibrium (0) and
    the damped-wave variant of Sec. 3.4 (1), with the same sizes; any other
    value is rejected on the host."""
    w = inputs.PIPE_D3Q19_SUB
    d0 = klb.desc_from_workload(w)
    d1 = klb.desc_from_workload(w.with_(phonon_wave=True))
    assert d0.phonon_eq == klb.KLB_PHONON_FLUID and d1.phonon_eq == klb.KLB_PHONON_WAVE
    assert klb.klb_lattice_bytes(d0) == klb.klb_lattice_bytes(d1) > 0
    d1.phonon_eq = 2
    assert klb.klb_lattice_bytes(d1) == 0
    with pytest.raises(klb.KLBError) as e:
        klb.klb_lattice_info(d1)
    assert e.value.status == 1 and "phonon_eq" in str(e.value)


def test_status_codes_match_the_header():
    """The binding's status names follow include/klb.h, including the
    saturated 16-bit range (KLB_ERANGE)."""
    import re

    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                            "klb.h")).read()
    body = hdr[hdr.index("typedef enum {\n    KLB_OK"):hdr.index("} klb_status;")]
    codes = {name: int(v) for name, v in re.findall(r"(KLB_[A-Z]+) = (\d+)", body)}
    for v, name in klb.STATUS.items():
        assert codes[name] == v, name
    assert codes["KLB_ERANGE"] == 7


def test_mask_geometry_and_empty_species():
    mask = np.array([[2, 1, 1, 2]], np.uint8)
    d = klb.make_desc(kind=9, nx=4, ny=4, nz=1, geom=klb.KLB_GEOM_MASK, mask=mask,
                      periodic_y=True)
    info = klb.klb_lattice_info(d)
    assert info["fluid_cs"] == 2 and info["solid_cs"] == 2 and math.isnan(info["d_wall"])
    d = klb.make_desc(kind=9, nx=4, ny=4, nz=1, geom=klb.KLB_GEOM_MASK,
                      mask=np.ones((1, 4), np.uint8), periodic_y=True)
    with pytest.raises(klb.KLBError, match="no solid"):
        klb.klb_lattice_info(d)


def test_reduced_storage_halves_the_population_footprint():
    w = inputs.PIPE_D3Q19_FP32
    b32 = klb.klb_lattice_bytes(klb.desc_from_workload(w))
    for st in ("fp16", "bf16"):
        b16 = klb.klb_lattice_bytes(klb.desc_from_workload(w.with_(storage=st)))
        assert b16 < 0.62 * b32


def _server(arena_bytes, storage=klb.KLB_FP32, **kw):
    """A server over a never-dereferenced arena address: creation, submission
    and counters are host logic and touch no device."""
    import ctypes

    lib = klb.load_library()
    o = klb.klb_server_opts(klb.KLB_D3Q19, storage, kw.get("check_every", 64),
                            kw.get("max_resident", 8), kw.get("autotune_steps", 0), 0)
    h = ctypes.c_void_p()
    st = lib.klb_server_create(ctypes.c_void_p(1 << 20), arena_bytes, None, ctypes.byref(o),
                               ctypes.byref(h))
    return lib, st, h


def test_server_host_logic_without_device():
    import ctypes

    lib, st, h = _server(1 << 20, autotune_steps=20, check_every=40)
    assert st == 1 and b"check_every" in lib.klb_server_last_error(None)
    tb = klb.klb_server_table_bytes(klb.KLB_FP32, 8)
    assert tb % 256 == 0 and tb > 0
    lib, st, h = _server(tb, max_resident=8)
    assert st == 2  # arena no larger than the table region
    w = inputs.PIPE_D3Q19_SUB
    need = klb.klb_lattice_bytes(klb.desc_from_workload(w))
    lib, st, h = _server(tb + need + 256)
    assert st == 0

    def req(w, **kw):
        return klb.klb_request(klb.desc_from_workload(w), klb.klb_couplings(*w.couplings),
                               kw.get("tol", 1e-9), kw.get("max_steps", 1000), 0.0,
                               kw.get("arrival", -1.0), kw.get("rid", 0))

    assert lib.klb_server_submit(h, ctypes.byref(req(w))) == 0
    assert lib.klb_server_submit(h, ctypes.byref(req(w, rid=1, arrival=5.0))) == 0
    big = w.with_(nx=2 * w.nx)
    assert lib.klb_server_submit(h, ctypes.byref(req(big))) == 1
    assert b"never fit" in lib.klb_server_last_error(h)
    assert lib.klb_server_submit(h, ctypes.byref(req(w.with_(storage="fp16")))) == 1
    assert lib.klb_server_submit(h, ctypes.byref(req(w, tol=0.0))) == 1
    assert lib.klb_server_submit(h, ctypes.byref(req(w, max_steps=0))) == 1
    assert lib.klb_server_submit(h, ctypes.byref(req(w.with_(tau=(0.5, 0.6, 1.0))))) == 1
    s = klb.klb_server_stats()
    assert lib.klb_server_get_stats(h, ctypes.byref(s)) == 0
    assert (s.queued, s.resident, s.finished, s.bytes_in_use) == (2, 0, 0, 0)
    assert s.table_bytes == tb and s.arena_bytes == tb + need + 256
    out = (klb.klb_result * 4)()
    assert lib.klb_server_poll(h, out, 4) == 0
    assert lib.klb_server_clock(h) >= 0.0
    assert lib.klb_server_destroy(h) == 0


def test_request_stream_recipe():
    rs = inputs.request_stream(200, rate=50.0, seed=0)
    gaps = np.diff([0.0] + [r.arrival for r in rs])
    assert np.all(gaps > 0) and 0.015 < gaps.mean() < 0.025
    for r in rs:
        w = r.w
        assert w.ny == w.nz and 32 ** 3 * 0.5 < w.nx * w.ny * w.nz < 512 * 128 * 128 * 1.5
        info = klb.klb_lattice_info(klb.desc_from_workload(w))
        assert info["active_sites"] > 0
    assert {r.w.geom for r in rs} == {"slab", "pipe"}


def test_normal_build_has_no_index_checks():
    assert klb.load_library().klb_bounds_checked() == 0


@pytest.mark.parametrize("change,msg", [
    (dict(nx=0), ">= 1"),
    (dict(ny=-2), ">= 1"),
    (dict(radius=0), "radius"),
    (dict(nx=65536, ny=2048, nz=2048, radius=900, shell=10), "32-bit"),
])
def test_degenerate_and_oversized_pipes_are_rejected(change, msg):
    d = klb.desc_from_workload(inputs.PIPE_D3Q19_FP32.with_(**change))
    assert klb.klb_lattice_bytes(d) == 0
    with pytest.raises(klb.KLBError, match=msg):
        klb.klb_lattice_info(d)


def test_lattices_beyond_32_bit_class_buffers():
    """Class buffers larger than 2^31 elements are admitted (row sources count
    in 32-element units, plane strides are 64-bit): a 4096 x 512 x 512 pipe
    (radius 240, shell 8) takes about 143 GB in FP32 and about half in FP16,
    its water buffer holding 19 x 181k rows x 4096 = 1.4e10 elements.  What
    stays 32-bit is one direction plane (rows x padded nx) and the box's cell
    number: a plane of 2^31 elements or more is refused."""
    w = inputs.PIPE_D3Q19_FP32.with_(nx=4096, ny=512, nz=512, radius=240, shell=8)
    b32 = klb.klb_lattice_bytes(klb.desc_from_workload(w))
    b16 = klb.klb_lattice_bytes(klb.desc_from_workload(w.with_(storage="fp16")))
    assert 1.2e11 < b32 < 1.6e11 and 0.45 * b32 < b16 < 0.6 * b32
    big_plane = w.with_(nx=3072, ny=1024, nz=1024, radius=480, storage="fp16")  # 723k rows x 3072
    assert klb.klb_lattice_bytes(klb.desc_from_workload(big_plane)) == 0
    with pytest.raises(klb.KLBError, match="row offsets"):
        klb.klb_lattice_info(klb.desc_from_workload(big_plane))


def test_serving_summary_statistics():
    """Latency = finish - arrival (queueing included), wait = admission -
    arrival, aggregate rate = site updates over the span from the first
    arrival to the last finish; unfinished requests are counted apart."""
    from paper_2403_15768_gb300 import serving

    def res(rid, arrival, admitted, finished, sites, steps, status=0):
        return {"id": rid, "arrival": arrival, "admitted": admitted, "finished": finished,
                "sites": sites, "steps": steps, "status": status}

    rs = [res(k, 0.1 * k, 0.1 * k + 0.01 * k, 0.1 * k + 1.0 + k, 1000, 100 * (k + 1)) for k in range(10)]
    rs[3]["status"] = 5
    s = serving.summarise({"results": rs + [None]})
    lat = np.array([1.0 + k for k in range(10)])
    wait = np.array([0.01 * k for k in range(10)])
    assert s["finished"] == 10 and s["submitted"] == 11
    assert s["p50_s"] == pytest.approx(np.percentile(lat, 50)) and s["p99_s"] == pytest.approx(np.percentile(lat, 99))
    assert s["wait_p99_s"] == pytest.approx(np.percentile(wait, 99))
    span = (0.9 + 1.0 + 9) - 0.0
    assert s["makespan_s"] == pytest.approx(span)
    assert s["mlups"] == pytest.approx(sum(1000 * 100 * (k + 1) for k in range(10)) / span / 1e6)
    assert s["status"] == {"KLB_OK": 9, "KLB_ETIMEOUT": 1}
    assert serving.summarise({"results": [None]}) == {"finished": 0}


def test_design_grid_recipe():
    """One pipe per (radius, g_we): box side 2 (radius + shell) + 2, the
    fixed couplings, net wall friction for a steady state, and every point a
    valid lattice."""
    ws = inputs.design_grid([6, 8, 12], [-0.02, 0.0, 0.05], nx=8, shell=3)
    assert len(ws) == 9
    for w in ws:
        assert w.geom == "pipe" and w.nx == 8 and w.ny == w.nz == 2 * (w.radius + w.shell) + 2
        g_we, g_wp = w.couplings[0], w.couplings[1]
        assert g_we + g_wp > 0  # a steady state exists
        assert klb.klb_lattice_bytes(klb.desc_from_workload(w)) > 0
    assert sorted({w.radius for w in ws}) == [6, 8, 12]
    assert sorted({w.couplings[0] for w in ws}) == [-0.02, 0.0, 0.05]


def test_perturbation_recipe():
    """drho = rho0 eps xi, u = eps eta, xi and eta uniform on (-1, 1) from
    default_rng(seed) in that order, box layout; no z velocity on D2Q9."""
    w = inputs.SLAB_D2Q9_FP64
    d, u = inputs.perturbation(w, 7, 1e-3)
    rng = np.random.default_rng(7)
    xi = rng.uniform(-1.0, 1.0, (3, w.nz, w.ny, w.nx))
    eta = rng.uniform(-1.0, 1.0, (3, 3, w.nz, w.ny, w.nx))
    assert d.shape == (3, w.nz, w.ny, w.nx) and u.shape == (3, 3, w.nz, w.ny, w.nx)
    assert np.array_equal(d, w.rho0 * 1e-3 * xi)
    assert np.array_equal(u[:, :2], 1e-3 * eta[:, :2]) and not u[:, 2].any()
    d3, u3 = inputs.perturbation(inputs.PIPE_D3Q19_SUB, 7, 1e-3)
    assert np.abs(u3[:, 2]).max() > 0 and np.abs(d3).max() <= 1e-3


def test_channel_sweep_recipe():
    """96 channels: slab or pipe (about half each), nx in [64, 512], box
    sides in [16, 128] (a pipe's box widened to fit its shell), shell in
    [2, 8], tau_w in [0.55, 1.2], drive in [1e-7, 1e-5], couplings in
    [1e-4, 1e-1] with g_ec = 0, and every channel inside the interface
    stability bound (at most two solid faces per fluid cell)."""
    ws = inputs.channel_sweep(96, seed=0)
    assert len(ws) == 96 and 30 <= sum(w.geom == "pipe" for w in ws) <= 66
    for w in ws:
        assert 64 <= w.nx <= 512 and 2 <= w.shell <= 8 and 16 <= w.nz <= 128
        assert 0.55 <= w.tau[0] <= 1.2 and w.tau[1:] == (0.6, 1.0)
        assert 1e-7 <= w.G[0] <= 1e-5 and w.G[1:] == (0.0, 0.0)
        g_we, g_wp, g_ep, g_ec, g_pc = w.couplings
        assert g_ec == 0.0 and all(1e-4 <= g <= 1e-1 for g in (g_we, g_wp, g_ep, g_pc))
        info = klb.klb_lattice_info(klb.desc_from_workload(w))
        assert info["max_faces"][0] <= 2
        assert info["max_faces"][0] * (g_we + g_wp) < 0.6 * w.rho0
    assert inputs.channel_sweep(96, seed=0) == ws and inputs.channel_sweep(96, seed=1) != ws
