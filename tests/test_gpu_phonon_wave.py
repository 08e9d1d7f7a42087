"""GPU parity of the phonon damped-wave variant (Sec. 3.4: phonons as linear
waves, d_tt n_p - cs^2 d_xx n_p = -gamma_p d_t n_p; KLB_PHONON_WAVE) against
the FP64 oracle, through the C ABI.

Tolerances as for the default scheme: FP64 1e-11 relative (operation order
and fused multiply-adds only); FP32 2e-4 of the field scale on short
perturbed runs and 1e-5 relative L2 after 10^4 steps; 16-bit storage 1e-3
(FP16) and 6e-3 (BF16) on short perturbed runs.  The single-mode test holds
the GPU to the closed form of the damped wave equation within the lattice's
O(k^2) correction, as the oracle pin does.
"""
import math

import numpy as np
import pytest

from klb_testutil import make_oracle, rel_l2, species_masks
from oracle import observables_from_fields
from paper_2403_15768_gb300 import inputs, klb

pytestmark = pytest.mark.gpu

SMALL_PIPE = inputs.PIPE_D3Q19_FP32.with_(name="pipe_r8_wave", nx=20, ny=24, nz=24, radius=8, shell=3,
                                          couplings=(0.05, 0.02, 0.1, 0.0, 0.01), phonon_wave=True)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    klb.load_library()


def _pair(w, seed, eps=1e-3):
    o = make_oracle(w)
    lat = klb.lattice_from_workload(w)
    d, u = inputs.perturbation(w, seed, eps)
    o.init_equilibrium(d, u)
    lat.init_equilibrium(d, u)
    return o, lat


@pytest.mark.parametrize("storage,tol", [("fp64", 1e-11), ("fp32", 2e-4), ("fp16", 1e-3), ("bf16", 6e-3)])
@pytest.mark.parametrize("case", ["pipe", "slab3d", "d2q9"])
def test_short_runs_against_oracle(case, storage, tol):
    """Perturbed start, 1 + 2 + 50 steps, every species' fields; in FP64 the
    phonon fields also differ from the default scheme's (the variant is
    active: its u u terms are about 1e-3 of the fields here)."""
    w = {
        "pipe": SMALL_PIPE.with_(nx=37),
        "slab3d": SMALL_PIPE.with_(geom="slab", nx=70, ny=14, nz=3, width=6, shell=3),
        "d2q9": inputs.SLAB_D2Q9_FP64.with_(phonon_wave=True),
    }[case].with_(storage=storage)
    if case == "d2q9" and storage != "fp64":
        w = w.with_(nx=66)
    o, lat = _pair(w, seed=7)
    for n in (1, 2, 50):
        o.step(n)
        lat.step(n)
    f = o.observe()
    drho, u = lat.get_field()
    masks = species_masks(o.geo, w.nx)
    for s in range(3):
        m = masks[s]
        ref = f["u"][s][:, m]
        assert np.abs(u[s][:, m] - ref).max() <= tol * np.abs(ref).max(), s
        assert np.abs(drho[s][m] - f["drho"][s][m]).max() <= tol * max(np.abs(f["drho"][s][m]).max(), 1e-3)
    ob = lat.observables()
    ob_o = o.observables()
    assert ob["flow_rate"] == pytest.approx(ob_o["flow_rate"], rel=max(tol, 1e-10))
    if storage != "fp64":
        return
    # the default scheme's phonons differ far beyond the tolerance
    o2 = make_oracle(w.with_(phonon_wave=False))
    d, uu = inputs.perturbation(w, 7, 1e-3)
    o2.init_equilibrium(d, uu)
    o2.step(53)
    up2 = o2.observe()["u"][2][:, masks[2]]
    assert np.abs(up2 - f["u"][2][:, masks[2]]).max() > 10 * tol * np.abs(f["u"][2][:, masks[2]]).max()


def test_fp32_pipe_10k_steps_against_oracle():
    """FP32 pipe with wave phonons, 10^4 steps from a perturbed start:
    relative L2 of every species' velocity field within 1e-5, slip length
    within 0.1%."""
    w = SMALL_PIPE
    o, lat = _pair(w, seed=1)
    o.step(10_000)
    lat.step(10_000)
    f = o.observe()
    _, u = lat.get_field()
    masks = species_masks(o.geo, w.nx)
    errs = [rel_l2(u[s][:, masks[s]], f["u"][s][:, masks[s]]) for s in range(3)]
    print("wave fp32 10k", errs)
    assert max(errs) <= 1e-5, errs
    ob_o = observables_from_fields(o.geo, w.nx, w.rho0, f)
    ob = lat.observables()
    assert ob["slip_length"] == pytest.approx(ob_o["slip_length"], rel=1e-3)
    assert ob["flow_rate"] == pytest.approx(ob_o["flow_rate"], rel=1e-5)


def _damped_mode_fit(a):
    """Decay rate and angular frequency of a sampled damped oscillation, from
    the three-term recurrence it satisfies (Prony's method)."""
    M = np.stack([a[1:-1], a[:-2]], 1)
    p, *_ = np.linalg.lstsq(M, a[2:], rcond=None)
    r = math.sqrt(-p[1])
    return -math.log(r), math.acos(p[0] / (2 * r))


def test_single_mode_damped_wave_closed_form():
    """A density mode of the phonons in a solid row (one fluid row beside it,
    no interface friction, so the phonons see only specular walls) decays at
    (gamma + 2 nu k^2)/2 and oscillates at sqrt(cs^2 k^2 - decay^2), with
    gamma = 2 atanh(gamma_pC/2) for the trapezoidal sink, on the GPU in FP64,
    and equals the oracle's run."""
    nx, gpc, tau_p = 256, 0.005, 1.0
    mask = np.array([[1, 2]], np.uint8)
    w = inputs.Workload(name="phonon_chain", kind=19, geom="mask", nx=nx, ny=2, nz=1,
                        tau=(0.8, 0.6, tau_p), G=(0.0, 0.0, 0.0), couplings=(0.0, 0.0, 0.0, 0.0, gpc),
                        storage="fp64", phonon_wave=True,
                        extra={"mask": mask, "periodic_y": True, "periodic_z": True})
    k = 2 * math.pi / nx
    x = np.arange(nx)
    drho = np.zeros((3, 1, 2, nx))
    drho[2, 0, 1] = 1e-6 * np.cos(k * x)
    u = np.zeros((3, 3, 1, 2, nx))
    lat = klb.lattice_from_workload(w)
    lat.init_equilibrium(drho, u)
    o = make_oracle(w)
    o.init_equilibrium(drho, u)
    amp = []
    for n in range(2000):
        lat.step(1)
        d, _ = lat.get_field()
        amp.append(d[2, 0, 1] @ np.cos(k * x) * 2 / nx)
        if n in (99, 1999):
            o.step(100 if n == 99 else 1900)
            assert np.abs(d[2] - o.observe()["drho"][2]).max() <= 1e-11 * 1e-6
    decay, freq = _damped_mode_fit(np.array(amp[50:]))
    nu = (tau_p - 0.5) / 3
    decay_th = (2 * math.atanh(gpc / 2) + 2 * nu * k * k) / 2
    freq_th = math.sqrt(k * k / 3 - decay_th ** 2)
    assert decay == pytest.approx(decay_th, rel=1e-4)
    assert freq == pytest.approx(freq_th, rel=3e-4)


def test_wave_lattice_in_a_batch_is_bitwise():
    """A lattice with wave phonons steps bit-identically alone and as a batch
    member next to a default lattice."""
    wa = SMALL_PIPE.with_(nx=45, storage="fp32")
    wb = wa.with_(phonon_wave=False, nx=33)
    alone = klb.lattice_from_workload(wa)
    a = klb.lattice_from_workload(wa)
    b = klb.lattice_from_workload(wb)
    d, u = inputs.perturbation(wa, 2, 1e-3)
    for lat in (alone, a):
        lat.init_equilibrium(d, u)
    batch = klb.Batch([a, b])
    batch.step(25)
    alone.step(25)
    for x, y in zip(alone.get_state(), a.get_state()):
        assert np.array_equal(x, y)
    batch.close()
