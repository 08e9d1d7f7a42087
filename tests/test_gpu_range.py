"""The range guard of 16-bit storage: a population difference from its row's
x-average beyond the representable range is stored saturated (the largest
finite 16-bit magnitude, not infinity), counted by the observation pass and
reported as KLB_ERANGE; values inside the range are stored exactly as
before.  The large perturbations are staged from the host."""
import numpy as np
import pytest

from paper_2403_15768_gb300 import inputs, klb

pytestmark = pytest.mark.gpu

PIPE = inputs.PIPE_D3Q19_FP32.with_(name="pipe_r8_range", nx=40, ny=24, nz=24, radius=8, shell=3,
                                    couplings=(0.05, 0.02, 0.1, 0.0, 0.01))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    klb.load_library()


def _alternating_density(w, amp):
    """Water density deviation +-amp alternating along x (row average 0):
    the rest population's difference from its row average is amp / 3."""
    d = np.zeros((3, w.nz, w.ny, w.nx))
    d[0] = amp * np.where(np.arange(w.nx) % 2 == 0, 1.0, -1.0)
    return d


def test_fp16_difference_beyond_range_is_saturated_and_reported():
    """FP16 differences are scaled by 2^20, so |g - ref| must stay below
    65504 * 2^-20 = 0.0625.  A +-0.3 density alternation puts the rest
    population of every water cell at 0.1 from its row average: every water
    cell holds one saturated population, the state stays finite, and the
    observables report KLB_ERANGE with the exact count.  (A few steps later
    the alternation has spread over the other populations and nothing is
    clipped any more; the state stays finite.)"""
    w = PIPE.with_(storage="fp16")
    lat = klb.lattice_from_workload(w)
    lat.init_equilibrium(_alternating_density(w, 0.3), None)
    with pytest.raises(klb.KLBError) as e:
        lat.observables()
    assert e.value.status == 7
    ob = lat.observables(allow_unstable=True)
    assert ob["clipped"] == lat.species_cells(0)
    assert ob["nonfinite"] == 0
    g, _, _ = lat.get_state()
    assert np.isfinite(g).all()
    rest = g[0, 0][:, :, 0]  # x = 0, drho = +0.3: saturated at ref + 65504 * 2^-20
    fluid = rest != 0
    assert np.allclose(rest[fluid], 65504.0 * 2.0 ** -20, rtol=0, atol=1e-7)
    lat.step(3)  # the saturated state steps on, finite
    ob = lat.observables(allow_unstable=True)
    assert ob["nonfinite"] == 0


def test_fp16_difference_inside_range_is_not_clipped():
    """+-0.18 puts the rest population at 0.06 from its row average, inside
    the FP16 range: nothing is clipped and the observables return KLB_OK."""
    w = PIPE.with_(storage="fp16")
    lat = klb.lattice_from_workload(w)
    lat.init_equilibrium(_alternating_density(w, 0.18), None)
    ob = lat.observables()
    assert ob["clipped"] == 0 and ob["nonfinite"] == 0
    g, _, _ = lat.get_state()
    rest = g[0, 0][:, :, 0]
    fluid = rest != 0
    assert np.allclose(rest[fluid], 0.06, rtol=2.0 ** -11)


def test_bf16_and_fp32_hold_the_same_perturbation():
    """BF16 (scale 1, range 3.4e38) and FP32 store the +-0.3 alternation
    without clipping."""
    for storage in ("bf16", "fp32"):
        w = PIPE.with_(storage=storage)
        lat = klb.lattice_from_workload(w)
        lat.init_equilibrium(_alternating_density(w, 0.3), None)
        ob = lat.observables()
        assert ob["clipped"] == 0 and ob["nonfinite"] == 0


def test_fp16_clipping_is_counted_per_species_cell():
    """The count is per species-cell: a +-0.3 alternation of the electron
    and phonon densities puts one saturated population in every solid cell
    of each species (2 x the solid cells), and water stays clear."""
    w = PIPE.with_(storage="fp16")
    lat = klb.lattice_from_workload(w)
    d = np.zeros((3, w.nz, w.ny, w.nx))
    alt = 0.3 * np.where(np.arange(w.nx) % 2 == 0, 1.0, -1.0)
    d[1] = alt
    d[2] = alt
    lat.init_equilibrium(d, None)
    ob = lat.observables(allow_unstable=True)
    assert ob["clipped"] == lat.species_cells(1) + lat.species_cells(2)
    assert ob["nonfinite"] == 0
