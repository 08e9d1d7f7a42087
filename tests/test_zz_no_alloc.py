"""klb_observables_static: the allocation-free observation entry point.

It exists for callers that cannot allocate device memory (an embedding host
owns the device allocator and hands out only the lattice buffer), so its
scratch lives in a static device array of the library.  Here it is called
through the C ABI and checked against klb_observables on the same lattice,
on two calls in a row, before and after further steps; lattices too large
for the static array must be rejected.  This file is collected last.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2403_15768_gb300 import inputs, klb

pytestmark = pytest.mark.gpu

RTOL = 1e-12  # same kernel and reduction order: results agree to round-off


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    klb.load_library()


def _static(lat):
    o = klb.klb_obs()
    st = klb.load_library().klb_observables_static(lat._h, ctypes.byref(o))
    return st, o.as_dict()


def _regular(lat):
    o = klb.klb_obs()
    st = klb.load_library().klb_observables(lat._h, ctypes.byref(o))
    return st, o.as_dict()


def _same(a, b):
    for k, v in a.items():
        w = b[k]
        for x, y in zip(np.atleast_1d(v), np.atleast_1d(w)):
            if isinstance(x, float) and math.isnan(x):
                assert math.isnan(y), k
            else:
                assert y == pytest.approx(x, rel=RTOL, abs=1e-300), k


@pytest.mark.parametrize("storage", ["fp32", "fp64"])
def test_static_observables_match_regular(storage):
    w = inputs.PIPE_D3Q19_FP32.with_(name="noalloc", nx=150, ny=24, nz=24, radius=8, shell=3,
                                     couplings=(0.05, 0.02, 0.1, 0.0, 0.01), storage=storage)
    lat = klb.lattice_from_workload(w)
    drho, u = inputs.perturbation(w, 5, 1e-3)
    lat.init_equilibrium(drho, u)
    lat.step(7)
    st, ref = _regular(lat)
    assert st == 0
    for _ in range(2):  # two calls in a row share the static array
        st, got = _static(lat)
        assert st == 0, klb.load_library().klb_last_error(lat._h)
        _same(ref, got)
    lat.step(5)
    st, ref = _regular(lat)
    st2, got = _static(lat)
    assert st == 0 and st2 == 0
    _same(ref, got)
    assert got["step"] == 12 and not math.isnan(got["residual"])


def test_static_observables_full_nanotube():
    w = inputs.PIPE_D3Q19_FP32
    lat = klb.lattice_from_workload(w)
    lat.step(10)
    st, ref = _regular(lat)
    for _ in range(2):
        st2, got = _static(lat)
        assert st == 0 and st2 == 0
        _same(ref, got)


def test_static_observables_reject_too_many_blocks():
    # 300 x 300 cross-section, one x plane: one observation block per cell
    mask = np.ones((300, 300), np.uint8)
    mask[:, 0] = 2
    w = inputs.Workload(name="wide", kind=19, geom="mask", nx=1, ny=300, nz=300,
                        extra={"mask": mask, "periodic_y": True, "periodic_z": True})
    lat = klb.lattice_from_workload(w)
    st, _ = _static(lat)
    assert st == 1
    msg = klb.load_library().klb_last_error(lat._h).decode()
    assert "KLB_STATIC_MAX_BLOCKS" in msg and str(klb.KLB_STATIC_MAX_BLOCKS) in msg
    st, _ = _regular(lat)
    assert st == 0
