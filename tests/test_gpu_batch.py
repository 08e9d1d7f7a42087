"""Batched stepping (klb_batch_*): many lattices of different sizes and
parameters advanced by one launch per step must give, bit for bit, what each
lattice gives stepped alone (a cell's update depends on its own lattice
only, and the block width changes no arithmetic), through graph replays of
whole periods, partial periods, reference refreshes of 16-bit storage and a
change of block width by the autotuner."""
import numpy as np
import pytest

from paper_2403_15768_gb300 import inputs, klb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    klb.load_library()


def _members(storage, n=5, seed=3):
    ws = inputs.channel_sweep(n, seed, storage=storage, scale=0.25)
    # one odd-sized member whose x extent is not a multiple of 32
    ws.append(inputs.PIPE_D3Q19_SUB.with_(name="odd", nx=37, ny=17, nz=15, radius=5, shell=2,
                                          storage=storage))
    return ws


def _perturbed(w, seed):
    lat = klb.lattice_from_workload(w)
    d, u = inputs.perturbation(w, seed, 1e-3)
    lat.init_equilibrium(d, u)
    return lat


def _same_state(a, b):
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("storage,steps", [("fp32", 20), ("fp16", 800), ("bf16", 70)])
def test_batch_equals_members_stepped_alone(storage, steps):
    ws = _members(storage)
    alone = [_perturbed(w, k) for k, w in enumerate(ws)]
    mates = [_perturbed(w, k) for k, w in enumerate(ws)]
    b = klb.Batch(mates)
    assert b.blocks > 0 and b.width in (32, 64, 128)
    b.step(steps // 2)
    b.step(steps - steps // 2)
    for lat in alone:
        lat.step(steps)
    for x, y in zip(alone, mates):
        assert y.nstep == steps
        _same_state(x, y)
        ox, oy = x.observables(), y.observables()
        assert ox["flow_rate"] == oy["flow_rate"] and ox["residual"] == oy["residual"]
    b.close()


def test_autotune_keeps_results_and_picks_a_width():
    ws = _members("fp32", n=3)
    alone = [_perturbed(w, k) for k, w in enumerate(ws)]
    mates = [_perturbed(w, k) for k, w in enumerate(ws)]
    b = klb.Batch(mates)
    width = b.autotune(steps_per_candidate=4)
    assert width in (32, 64, 128) and b.width == width
    taken = mates[0].nstep
    assert taken == 3 * (1 + 4)
    b.step(13)
    for lat in alone:
        lat.step(taken + 13)
    for x, y in zip(alone, mates):
        _same_state(x, y)


def test_fp64_d2q9_batch():
    ws = [inputs.SLAB_D2Q9_FP64.with_(nx=nx, width=wd, ny=wd + 8, tau=(t, 0.6, 1.0))
          for nx, wd, t in ((64, 32, 0.8), (40, 10, 0.6), (100, 21, 1.1))]
    alone = [_perturbed(w, k) for k, w in enumerate(ws)]
    mates = [_perturbed(w, k) for k, w in enumerate(ws)]
    b = klb.Batch(mates)
    b.step(15)
    for lat in alone:
        lat.step(15)
    for x, y in zip(alone, mates):
        _same_state(x, y)


def test_member_stepped_alone_leaves_the_batch():
    ws = _members("fp32", n=2)
    mates = [_perturbed(w, k) for k, w in enumerate(ws)]
    b = klb.Batch(mates)
    b.step(3)
    mates[1].step(1)
    with pytest.raises(klb.KLBError) as e:
        b.step(1)
    assert e.value.status == 6 and "outside the batch" in str(e.value)
    # observing a member does not take it out of phase
    b2 = klb.Batch(mates[:1])
    mates[0].observables()
    b2.step(2)
    assert mates[0].nstep == 5


def test_batch_rejects_mixed_members():
    a = _perturbed(_members("fp32", n=1)[0], 0)
    c = _perturbed(_members("fp16", n=1)[0], 0)
    with pytest.raises(klb.KLBError, match="kind and storage"):
        klb.Batch([a, c])
    with pytest.raises(klb.KLBError, match="twice"):
        klb.Batch([a, a])


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_members_at_different_time_levels(storage):
    """Members admitted at different times (steps 0, 7, 40 and 100, so that
    16-bit members need reference refreshes at different phases) batch
    together and still match their twins stepped alone, over more than one
    period of the step pattern."""
    ws = _members(storage, n=3)
    lead = [0, 7, 40, 100]
    alone = [_perturbed(w, k) for k, w in enumerate(ws[:4])]
    mates = [_perturbed(w, k) for k, w in enumerate(ws[:4])]
    for x, y, n in zip(alone, mates, lead):
        x.step(n)
        y.step(n)
    b = klb.Batch(mates)
    b.step(400)
    for x, n in zip(alone, lead):
        x.step(400)
    for x, y, n in zip(alone, mates, lead):
        assert y.nstep == n + 400
        _same_state(x, y)
