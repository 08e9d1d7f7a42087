"""GPU parity of reduced-precision storage (FP16 / BF16 differences from a
per-row FP32 reference, FP32 arithmetic) against the FP64 oracle, and the
full-size nanotube against the oracle.

Bars: the FP32 velocity field within 1e-5 relative L2 after 10^4 steps and
the slip length within 0.1%; flow rate and slip length within 1% for 16-bit
storage.  FP32 storage is held to 1e-6, ten times tighter: its fix-up adds
its increments with a dither of one ulp (unbiased rounding), which brought
the measured error from 3.6e-6-4.0e-6 to 0.9e-7-1.7e-7 on the full nanotube
and the subcase, and a bias coming back would show as a few 1e-6.  Where no bar is stated (16-bit velocity fields, the small cases),
tolerances are the errors measured on GB300 with a margin of about 2x
(small pipe after 10^4 steps: FP16 4.6e-6, BF16 2.5e-5; perturbed start
after 2000 steps: FP16 4.2e-4, BF16 2.6e-3).
"""
import numpy as np
import pytest

from klb_testutil import make_oracle, oracle_geometry, rel_l2, species_masks
from oracle import observables_from_fields
from paper_2403_15768_gb300 import inputs, klb

pytestmark = pytest.mark.gpu

SMALL_PIPE = inputs.PIPE_D3Q19_FP32.with_(name="pipe_r8", nx=20, ny=24, nz=24, radius=8, shell=3,
                                          couplings=(0.05, 0.02, 0.1, 0.0, 0.01))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    klb.load_library()


def _run_pair(w, storage, seed, steps, oracle_cache={}):
    key = (repr(w), seed, steps)
    if key not in oracle_cache:
        o = make_oracle(w)
        if seed is not None:
            d, u = inputs.perturbation(w, seed, 1e-3)
            o.init_equilibrium(d, u)
        else:
            o.init_equilibrium()
        o.step(steps)
        f = o.observe()
        oracle_cache[key] = (o.geo, f, observables_from_fields(o.geo, w.nx, w.rho0, f))
    geo, f, ob_o = oracle_cache[key]
    lat = klb.lattice_from_workload(w.with_(storage=storage))
    if seed is not None:
        d, u = inputs.perturbation(w, seed, 1e-3)
        lat.init_equilibrium(d, u)
    lat.step(steps)
    _, ug = lat.get_field()
    m = species_masks(geo, w.nx)
    errs = [rel_l2(ug[s][:, m[s]], f["u"][s][:, m[s]]) for s in range(3)]
    return errs, lat.observables(), ob_o


@pytest.mark.parametrize("storage,tol", [("fp16", 1e-5), ("bf16", 6e-5)])
def test_reduced_quiescent_10k_small_pipe(storage, tol):
    errs, ob, ob_o = _run_pair(SMALL_PIPE, storage, None, 10_000)
    assert max(errs) <= tol, errs
    assert ob["flow_rate"] == pytest.approx(ob_o["flow_rate"], rel=1e-5)
    assert ob["slip_length"] == pytest.approx(ob_o["slip_length"], rel=1e-3)


@pytest.mark.parametrize("storage,tol", [("fp16", 1e-3), ("bf16", 6e-3)])
def test_reduced_perturbed_start(storage, tol):
    errs, ob, ob_o = _run_pair(SMALL_PIPE, storage, 1, 2000)
    assert max(errs) <= tol, errs
    assert ob["flow_rate"] == pytest.approx(ob_o["flow_rate"], rel=1e-2)
    assert ob["slip_length"] == pytest.approx(ob_o["slip_length"], rel=1e-2)


@pytest.mark.parametrize("storage,tol", [("fp16", 2e-5), ("bf16", 5e-5)])
def test_reduced_d2q9_slab_10k(storage, tol):
    w = inputs.SLAB_D2Q9_FP64.with_(storage="fp32")
    errs, ob, ob_o = _run_pair(w, storage, None, 10_000)
    assert max(errs) <= tol, errs
    assert ob["slip_length"] == pytest.approx(ob_o["slip_length"], rel=1e-3)


_FULL = {}
FULL_STEPS = 10_000
# the bars: 0.1% for FP32, 1% for 16-bit storage
PER_OBS_TOL = {"fp32": 1e-3, "fp16": 1e-2, "bf16": 1e-2}


def _full_oracle():
    """Oracle of the 512x128x128 nanotube from rest, on one x plane: a
    quiescent start stays exactly x-invariant, so every x plane of the full
    lattice must equal it."""
    if not _FULL:
        w = inputs.PIPE_D3Q19_FP32
        o = make_oracle(w, nx=1)
        o.init_equilibrium()
        o.step(FULL_STEPS)
        f = o.observe()
        _FULL["geo"], _FULL["f"] = o.geo, f
        _FULL["obs"] = observables_from_fields(o.geo, 1, w.rho0, f)
    return _FULL["geo"], _FULL["f"], _FULL["obs"]


def _per_observable(ob, ob_o):
    keys = ("flow_rate", "slip_length", "u_slip", "dudn_wall", "u_wallrow_mean")
    err = {k: abs(ob[k] / ob_o[k] - 1.0) for k in keys}
    err.update({f"mean_u[{s}]": abs(ob["mean_u"][s] / ob_o["mean_u"][s] - 1.0) for s in range(3)})
    return err


@pytest.mark.parametrize("storage,tol", [("fp32", 1e-6), ("fp16", 1e-5), ("bf16", 1e-5)])
def test_full_nanotube_10k_steps_against_oracle(storage, tol):
    """The 512x128x128 nanotube in the benchmark's launch configuration, 10^4
    steps from rest, against the oracle: FP32 velocity fields within 1e-5
    relative L2 and slip length within 0.1%; every observable of the
    slip-length study within its bar."""
    import torch

    geo, f, ob_o = _full_oracle()
    w = inputs.PIPE_D3Q19_FP32.with_(storage=storage)
    lat = klb.lattice_from_workload(w)
    lat.step(FULL_STEPS)
    _, ug = lat.get_field()
    ob = lat.observables()
    m = species_masks(geo, 1)
    errs = []
    for s in range(3):
        assert np.abs(ug[s] - ug[s][..., :1]).max() == 0.0  # every x plane identical
        errs.append(rel_l2(ug[s][..., :1][:, m[s]], f["u"][s][:, m[s]]))
    per_obs = _per_observable(ob, ob_o)
    print(storage, "rel-L2", errs, per_obs)
    assert max(errs) <= tol, errs
    assert per_obs["slip_length"] <= PER_OBS_TOL[storage]
    assert per_obs["flow_rate"] <= 1e-4
    assert max(per_obs.values()) <= PER_OBS_TOL[storage], per_obs
    assert ob["nonfinite"] == 0 and ob["clipped"] == 0
    del lat
    torch.cuda.empty_cache()


_SUB = {}


def _sub_oracle():
    """The oracle's 128x64x64 subcase after 5000 steps from a perturbed,
    x-varying start, as stored by tests/golden/make_pipe_sub_oracle.py (the
    oracle needs about ten minutes of one core for it)."""
    if not _SUB:
        import json
        import os

        z = np.load(os.path.join(os.path.dirname(__file__), "golden", "pipe_sub_perturbed_5000.npz"))
        _SUB.update(steps=int(z["steps"]), seed=int(z["seed"]), eps=float(z["eps"]),
                    planes=[int(v) for v in z["planes"]], u=z["u"], drho=z["drho"],
                    obs=json.loads(str(z["observables"])))
    return _SUB


# the x-varying part (differences between the stored planes, about 3e-4 of
# the flow at step 5000) carries the 16-bit rounding of the stored
# differences; measured on GB300 2.2x below these: FP32 1.5e-4, FP16 1.7e-3,
# BF16 1.0e-1 (BF16 keeps 8 bits of a difference that is itself small)
XVAR_TOL = {"fp32": 3e-4, "fp16": 4e-3, "bf16": 0.2}


@pytest.mark.parametrize("storage,tol", [("fp32", 1e-6), ("fp16", 2e-5), ("bf16", 2e-3)])
def test_subcase_perturbed_start_against_oracle(storage, tol):
    """The 128x64x64 nanotube subcase (radius 24, shell 3) from a seeded,
    x-varying perturbed start, 5000 steps, against the FP64 oracle: velocity
    fields of every species on the stored x planes (relative L2), and every
    observable; flow rate and slip length within 1% for 16-bit storage,
    0.1% for FP32."""
    ref = _sub_oracle()
    w = inputs.PIPE_D3Q19_SUB.with_(storage=storage)
    lat = klb.lattice_from_workload(w)
    d, u = inputs.perturbation(w, ref["seed"], ref["eps"])
    lat.init_equilibrium(d, u)
    lat.step(ref["steps"])
    _, ug = lat.get_field()
    ob = lat.observables()
    geo = oracle_geometry(w)
    m = species_masks(geo, len(ref["planes"]))
    ug = ug[..., ref["planes"]]
    errs = [rel_l2(ug[s][:, m[s]], ref["u"][s][:, m[s]]) for s in range(3)]
    # the start really is x-varying, and still is at the end
    assert np.abs(ref["u"][0, 0, ..., 0] - ref["u"][0, 0, ..., 1]).max() > 1e-4 * np.abs(ref["u"][0, 0]).max()
    # the x-varying part alone: differences between the stored planes
    dx = [rel_l2((ug[s][..., 1:] - ug[s][..., :1])[:, m[s][..., 1:]],
                 (ref["u"][s][..., 1:] - ref["u"][s][..., :1])[:, m[s][..., 1:]]) for s in range(3)]
    per_obs = _per_observable(ob, ref["obs"])
    print(storage, "rel-L2", errs, "x-varying part", dx, per_obs)
    assert max(errs) <= tol, errs
    assert max(dx) <= XVAR_TOL[storage], dx
    bar = 1e-3 if storage == "fp32" else 1e-2
    assert per_obs["flow_rate"] <= bar and per_obs["slip_length"] <= bar, per_obs
    assert ob["nonfinite"] == 0 and ob["clipped"] == 0


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_reduced_state_roundtrip_and_one_step(storage):
    """klb_set_state encodes against the state's x-averages; reading it back
    returns each population within the 16-bit precision of its difference
    from that average; one step from the oracle's state matches the oracle."""
    w = SMALL_PIPE.with_(nx=40, storage=storage)
    o = make_oracle(w)
    d, u = inputs.perturbation(w, 3, 1e-3)
    o.init_equilibrium(d, u)
    o.step(20)
    g, U1, U2 = o.get_state()
    lat = klb.lattice_from_workload(w)
    lat.set_state(g, U1, U2, step=20)
    g_back, _, _ = lat.get_state()
    # g_back = f32(s16((f32(g) - ref) * 2^k) / 2^k + ref), ref = f32(mean over x):
    # the 16-bit rounding of the difference plus three FP32 roundings of g.
    dev = g - g.mean(axis=-1, keepdims=True)
    rel = 2.0 ** -11 if storage == "fp16" else 2.0 ** -8
    eps32 = 2.0 ** -24
    bound = rel * (np.abs(dev) + eps32 * np.abs(g).max()) + 4 * eps32 * np.abs(g) + 1e-13
    assert np.all(np.abs(g_back - g) <= bound)
    o.step(1)
    lat.step(1)
    _, ug = lat.get_field()
    f = o.observe()
    m = species_masks(o.geo, w.nx)
    for s in range(3):
        assert rel_l2(ug[s][:, m[s]], f["u"][s][:, m[s]]) <= (1e-3 if storage == "fp16" else 6e-3)
