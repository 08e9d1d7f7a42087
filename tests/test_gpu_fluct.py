"""Thermal fluctuations of the water (klb_set_fluctuations; Eq. 6, Eq. 17):
the GPU draws the same Philox-4x32-10 words as the oracle, so the noisy
fields match it element by element (FP64 to rounding, FP32 within the
precision of its single-precision Box-Muller), and the lattice fluid obeys
equipartition, rho0 <u_a^2> = kT, <drho^2> = rho0 kT / cs^2."""
import numpy as np
import pytest

from klb_testutil import make_oracle, species_masks
from paper_2403_15768_gb300 import inputs, klb

pytestmark = pytest.mark.gpu

KT, SEED = 1e-5, 0x5EED_1234_ABCD


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    klb.load_library()


def _noisy_pair(w, steps):
    o = make_oracle(w)
    o.init_equilibrium()
    o.set_fluctuations(KT, SEED)
    lat = klb.lattice_from_workload(w)
    lat.set_fluctuations(KT, SEED)
    o.step(steps)
    lat.step(steps)
    return o, lat


PIPE = inputs.PIPE_D3Q19_FP32.with_(nx=24, ny=24, nz=24, radius=8, shell=3)


@pytest.mark.parametrize("w,steps,rtol", [
    (inputs.SLAB_D2Q9_FP64.with_(nx=40), 25, 1e-10),
    (PIPE.with_(storage="fp64"), 10, 1e-10),
    (PIPE, 10, 2e-4),
], ids=["d2q9_fp64", "d3q19_fp64", "d3q19_fp32"])
def test_noise_matches_oracle(w, steps, rtol):
    o, lat = _noisy_pair(w, steps)
    f = o.observe()
    drho, u = lat.get_field()
    m = species_masks(o.geo, w.nx)
    for s in range(3):
        ref, got = f["u"][s][:, m[s]], u[s][:, m[s]]
        assert np.abs(got - ref).max() <= rtol * np.abs(ref).max(), s
        dr, dg = f["drho"][s][m[s]], drho[s][m[s]]
        assert np.abs(dg - dr).max() <= rtol * max(np.abs(dr).max(), 1e-12), s
    assert np.abs(f["u"][0][0][m[0]]).max() > 1e-4  # thermal, not the drive alone


@pytest.mark.parametrize("storage", ["fp32", "fp64"])
def test_equipartition_on_gpu(storage):
    w = inputs.SLAB_D2Q9_FP64.with_(kind=19, nx=64, ny=24, nz=8, width=16, shell=4, G=(0.0, 0.0, 0.0),
                                    couplings=(0.0,) * 5, storage=storage)
    lat = klb.lattice_from_workload(w)
    lat.set_fluctuations(KT, 77)
    lat.step(500)
    fluid = np.zeros((w.nz, w.ny), bool)
    fluid[:, 4:20] = True
    acc = np.zeros(4)
    n = 150
    for _ in range(n):
        lat.step(5)
        drho, u = lat.get_field()
        m = np.broadcast_to(fluid[..., None], drho[0].shape)
        acc += [np.mean(u[0][0][m] ** 2), np.mean(u[0][1][m] ** 2), np.mean(u[0][2][m] ** 2),
                np.mean(drho[0][m] ** 2)]
    acc /= n
    for a in range(3):
        assert acc[a] == pytest.approx(KT, rel=0.03), acc / KT
    assert acc[3] == pytest.approx(3 * KT, rel=0.03)


def test_noise_off_and_rejections():
    a, b = klb.lattice_from_workload(PIPE), klb.lattice_from_workload(PIPE)
    b.set_fluctuations(KT, 1)
    b.set_fluctuations(0.0, 1)  # off again
    a.step(7)
    b.step(7)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    b.set_fluctuations(KT, 1)
    with pytest.raises(klb.KLBError, match="batched"):
        klb.Batch([a, b])
    h = klb.lattice_from_workload(PIPE.with_(storage="fp16"))
    with pytest.raises(klb.KLBError, match="FP32 or FP64"):
        h.set_fluctuations(KT, 1)
    with pytest.raises(klb.KLBError, match="kT"):
        a.set_fluctuations(-1.0, 1)
