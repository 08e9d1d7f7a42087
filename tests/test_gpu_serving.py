"""The request loop (klb_server_*): each request's result is the same alone
and in a mix with others admitted before, with and after it (bit for bit:
every resident lattice advances a fixed number of steps per round and is
checked at multiples of it since its own admission); admission respects the
arena; step limits and non-finite states retire requests with their
status."""
import numpy as np
import pytest

from paper_2403_15768_gb300 import inputs, klb, serving

pytestmark = pytest.mark.gpu

STREAM = inputs.request_stream(7, rate=50.0, seed=5, min_cells=6 ** 3, max_cells=20 ** 3)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    klb.load_library()


def _bytes(w):
    return klb.klb_lattice_bytes(klb.desc_from_workload(w))


def _run(reqs, arena, storage="fp32", check_every=20, autotune_steps=0, tol=1e-8,
         max_steps=2000, stagger=False):
    srv = klb.Server(arena, storage=storage, check_every=check_every, max_resident=8,
                     autotune_steps=autotune_steps)
    out = {}
    pending = list(reqs)
    it = 0
    while pending or len(out) < len(reqs):
        # staggered: one new request every second round
        it += 1
        if pending and (not stagger or it % 2 == 1):
            r = pending.pop(0)
            srv.submit(klb.desc_from_workload(r.w), r.w.couplings, tol, max_steps, r.rid)
        srv.tick()
        for res in srv.poll():
            out[res["id"]] = res
    stats = srv.stats()
    srv.close()
    return out, stats


def _same(a, b):
    assert a["status"] == b["status"] and a["steps"] == b["steps"]
    for k, v in a["obs"].items():
        w = b["obs"][k]
        assert np.array_equal(np.asarray(v), np.asarray(w), equal_nan=True), k


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_result_alone_equals_result_in_the_mix(storage):
    reqs = [inputs.Request(r.rid, r.arrival, r.w.with_(storage=storage)) for r in STREAM]
    total = sum(_bytes(r.w) for r in reqs)
    arena = total + klb.klb_server_table_bytes(klb.STORAGE[storage], 8) + 64 * 1024 * 1024
    tol = 1e-8 if storage == "fp32" else 1e-6
    alone = {r.rid: _run([r], arena, storage, tol=tol)[0][r.rid] for r in reqs}
    mix, stats = _run(reqs, arena, storage, tol=tol, stagger=True, autotune_steps=2)
    assert stats["batch_forms"] >= 3 and stats["finished"] == len(reqs)
    assert stats["peak_bytes_in_use"] <= arena
    for r in reqs:
        _same(alone[r.rid], mix[r.rid])
        assert mix[r.rid]["steps"] % 20 == 0
    assert any(v["status"] == 0 for v in mix.values())


def test_admission_waits_for_arena_space():
    """An arena that holds the two largest requests only: requests queue,
    the peak footprint stays inside the arena, and results are unchanged."""
    sizes = sorted((_bytes(r.w) for r in STREAM), reverse=True)
    arena = klb.klb_server_table_bytes(klb.KLB_FP32, 8) + sizes[0] + sizes[1] + 4096
    small, stats = _run(STREAM, arena)
    big, _ = _run(STREAM, 4 * sum(sizes))
    assert stats["peak_bytes_in_use"] <= sizes[0] + sizes[1] + 4096
    for r in STREAM:
        _same(small[r.rid], big[r.rid])
        assert small[r.rid]["admitted"] >= small[r.rid]["arrival"]


def test_step_limit_and_unstable_requests():
    """A drive of 1e30 overflows FP32 velocities in the first step; the
    request is retired as unstable at its first check."""
    w = STREAM[0].w
    blow = w.with_(G=(1e30, 0.0, 0.0))
    reqs = [inputs.Request(0, 0.0, w), inputs.Request(1, 0.0, blow)]
    out, _ = _run(reqs, 4 * (_bytes(w) + 2 ** 26), check_every=64, tol=1e-30, max_steps=100)
    assert out[0]["status"] == 5 and out[0]["steps"] == 128  # KLB_ETIMEOUT at the first check >= 100
    assert out[1]["status"] == 4 and out[1]["obs"]["nonfinite"] > 0  # KLB_EUNSTABLE
    assert out[1]["steps"] == 64


def test_replay_reports_latencies():
    srv = klb.Server(256 * 1024 * 1024, check_every=25, max_resident=8)
    run = serving.replay(srv, STREAM, tol=1e-8, max_steps=300)
    s = serving.summarise(run)
    srv.close()
    assert s["finished"] == len(STREAM) and s["p99_s"] >= s["p50_s"] > 0 and s["mlups"] > 0
    for r in run["results"]:
        assert r["arrival"] <= r["admitted"] <= r["finished"]


def test_design_map_matches_oracle_steady_states():
    """A small design map (pipes of radius 6 and 8, water-electron friction
    -0.02 and +0.05) run to steady state through the request loop in FP64
    equals the oracle's steady states: slip length, flow rate and electron
    wind."""
    from klb_testutil import make_oracle
    from oracle import observables_from_fields

    ws = inputs.design_grid([6, 8], [-0.02, 0.05], nx=2, shell=2, storage="fp64")
    srv = klb.Server(64 * 1024 * 1024, storage="fp64", check_every=500, max_resident=8)
    res = serving.design_map(srv, ws, tol=1e-16, max_steps=300_000)
    srv.close()
    for w, r in zip(ws, res):
        assert r["status"] == 0, r
        o = make_oracle(w, nx=1)
        o.init_equilibrium()
        prev = None
        for _ in range(150):
            o.step(2000)
            f = o.observe()
            if prev is not None and np.abs(f["u"] - prev).max() < 1e-14 * np.abs(f["u"]).max():
                break
            prev = f["u"]
        else:
            raise AssertionError("oracle not steady")
        ob = observables_from_fields(o.geo, 1, w.rho0, f)
        assert r["slip_length"] == pytest.approx(ob["slip_length"], rel=1e-6)
        assert r["flow_rate"] == pytest.approx(ob["flow_rate"], rel=1e-7)
        ue = f["u"][1][0][species_solid(o.geo)].mean()
        assert r["mean_u_e"] == pytest.approx(ue, rel=1e-6)
    # the negative coupling changes the slip: the map is not flat in g_we
    assert res[0]["slip_length"] != pytest.approx(res[1]["slip_length"], rel=1e-3)


def species_solid(geo):
    return np.broadcast_to((geo.cs_type == 2)[:, :, None], (geo.nz, geo.ny, 1))
