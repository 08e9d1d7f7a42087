"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test states an independent fact (a closed form, a conservation law, an
identity of the lattice, an independent dense solve, a symmetry) so that a
plausible mistake in the oracle -- a dropped term, a wrong sign or index, a
transposed operand -- fails at least one of them.  No expected value comes
from the CUDA path.
"""
import math
import os

import numpy as np
import pytest

from oracle import Oracle, cross_section, slip_poiseuille_pipe, slip_poiseuille_slab
from oracle.oracle import T_FLUID, T_SOLID

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CS2 = 1.0 / 3.0


def _slab(Q=9, nx=1, ny=40, width=32, shell=4, **kw):
    nz = 1
    geo = cross_section("slab", ny, nz, width=width, shell=shell)
    return Oracle(Q, nx, geo, **kw), geo


def _mask(Q, nx, rows, periodic_y=True, **kw):
    """Cross-section from a list of row types (z-invariant, one z plane)."""
    t = np.array(rows, np.uint8)[None, :]
    geo = cross_section("mask", len(rows), 1, mask=t, periodic_y=periodic_y, periodic_z=True)
    return Oracle(Q, nx, geo, **kw), geo


def _run_to_steady(o, tol=1e-15, chunk=2000, max_steps=400000):
    prev = None
    n = 0
    while n < max_steps:
        o.step(chunk)
        n += chunk
        u = o.observe()["u"]
        if prev is not None and np.abs(u - prev).max() < tol:
            return u
        prev = u
    raise AssertionError("no steady state")


# ---------------------------------------------------------------------------
# Lattice tables (Sec. 4: D2Q9 numbering printed in Sec. 4.2)

def test_d2q9_numbering_matches_paper():
    o, _ = _slab()
    c, w, opp = o.lattice()
    fixture = {}
    with open(os.path.join(GOLDEN, "d2q9_numbering.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                i, cx, cy = map(int, line.split())
                fixture[i] = (cx, cy)
    for i in range(9):
        assert tuple(c[i, :2]) == fixture[i]
        assert c[i, 2] == 0


@pytest.mark.parametrize("Q", [9, 19])
def test_lattice_isotropy(Q):
    o = _slab(Q)[0] if Q == 9 else Oracle(19, 1, cross_section("pipe", 8, 8, radius=2, shell=1))
    c, w, opp = o.lattice()
    d = 2 if Q == 9 else 3
    c = c[:, :d].astype(float)
    assert len({tuple(v) for v in c}) == Q
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(w @ c).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib->ab", w, c, c) - CS2 * np.eye(d)).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib,ic->abc", w, c, c, c)).max() < 1e-15
    I = np.eye(d)
    iso4 = CS2 ** 2 * (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
                       + np.einsum("ad,bc->abcd", I, I))
    assert np.abs(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c) - iso4).max() < 1e-15
    for i in range(Q):
        assert np.array_equal(c[opp[i]], -c[i])


# ---------------------------------------------------------------------------
# P1: moment identities of the equilibrium and of the Guo source

@pytest.mark.parametrize("Q", [9, 19])
def test_moment_identities(Q):
    if Q == 9:
        o = _slab()[0]
    else:
        o = Oracle(19, 1, cross_section("pipe", 8, 8, radius=2, shell=1))
    c, w, _ = o.lattice()
    rng = np.random.default_rng(7)
    for _ in range(5):
        drho = rng.uniform(-0.05, 0.05)
        rho = 1.0 + drho
        u = rng.uniform(-0.05, 0.05, 3)
        F = rng.uniform(-1e-3, 1e-3, 3)
        if Q == 9:
            u[2] = F[2] = 0.0
        om = rng.uniform(0.6, 1.9)
        eq = np.array([o.geq(i, drho, u) for i in range(Q)])
        S = np.array([o.guo(i, om, u, F) for i in range(Q)])
        cf = c.astype(float)
        d = 2 if Q == 9 else 3
        I = np.eye(3)
        I[d:, d:] = 0
        assert abs(eq.sum() - drho) < 1e-15
        assert np.abs(cf.T @ eq - rho * u).max() < 1e-15
        P = np.einsum("i,ia,ib->ab", eq, cf, cf)
        assert np.abs(P - (drho * CS2 * I + rho * np.outer(u, u))).max() < 1e-15
        assert abs(S.sum()) < 1e-16
        assert np.abs(cf.T @ S - (1 - om / 2) * F).max() < 1e-16
        PS = np.einsum("i,ia,ib->ab", S, cf, cf)
        assert np.abs(PS - (1 - om / 2) * (np.outer(u, F) + np.outer(F, u))).max() < 1e-16


# ---------------------------------------------------------------------------
# Streaming / boundary rule (Sec. 4.2)

def _geometries():
    yield 9, 6, cross_section("slab", 40, 1, width=32, shell=4)
    yield 19, 5, cross_section("slab", 14, 3, width=6, shell=3)
    yield 19, 4, cross_section("pipe", 26, 26, radius=9, shell=3)
    yield 19, 3, cross_section("pipe", 17, 15, radius=5, shell=2)
    yield 19, 3, cross_section("pipe", 12, 12, radius=3, shell=1)


@pytest.mark.parametrize("bb", [False, True])
def test_streaming_is_a_permutation(bb):
    """Every post-collision population is pulled exactly once: the map
    (cell, i) -> (source cell, source direction) is a bijection per species
    (this is what makes the scheme conserve mass)."""
    for Q, nx, geo in _geometries():
        o = Oracle(Q, nx, geo, iface_bounceback=bb)
        for s in range(3):
            src, sd = o.stream_table(s)
            live = src >= 0
            keys = src[live] * Q + sd[live]
            assert len(np.unique(keys)) == keys.size
            assert keys.size == live.sum()
            owners = np.flatnonzero(live.any(axis=0))
            assert set(np.unique(src[live])) <= set(owners)


def test_flat_wall_rules_d2q9():
    """Slab rows 0-3 solid, 4-35 fluid, 36-39 solid.  Specular at the
    liquid/solid interface for all species, bounce-back at the outer faces."""
    nx = 6
    o, geo = _slab(nx=nx)
    N = o.ncell
    cell = lambda x, y: (x % nx) + nx * y  # noqa: E731
    src, sd = o.stream_table(0)
    E, Nn, W, S, NE, NW, SW, SE = 1, 2, 3, 4, 5, 6, 7, 8
    x, y = 2, 4  # bottom wall row of the fluid
    assert (src[Nn, cell(x, y)], sd[Nn, cell(x, y)]) == (cell(x, y), S)
    assert (src[NE, cell(x, y)], sd[NE, cell(x, y)]) == (cell(x - 1, y), SE)
    assert (src[NW, cell(x, y)], sd[NW, cell(x, y)]) == (cell(x + 1, y), SW)
    assert (src[E, cell(x, y)], sd[E, cell(x, y)]) == (cell(x - 1, y), E)
    y = 35  # top wall row
    assert (src[SE, cell(x, y)], sd[SE, cell(x, y)]) == (cell(x - 1, y), NE)
    srce, sde = o.stream_table(1)
    y = 3  # top solid row of the bottom wall: interface above
    assert (srce[SW, cell(x, y)], sde[SW, cell(x, y)]) == (cell(x + 1, y), NW)
    y = 0  # outer face below
    assert (srce[NE, cell(x, y)], sde[NE, cell(x, y)]) == (cell(x, y), SW)
    assert (srce[Nn, cell(x, y)], sde[Nn, cell(x, y)]) == (cell(x, y), S)
    assert N == nx * 40


def test_specular_links_keep_cx():
    """Specular links never reverse c_x, so they exchange no x-momentum; links
    that reverse c_x are exactly the bounce-back ones (same cell, opposite
    direction)."""
    for Q, nx, geo in _geometries():
        o = Oracle(Q, nx, geo)
        c, _, opp = o.lattice()
        for s in range(3):
            src, sd = o.stream_table(s)
            for i in range(Q):
                live = src[i] >= 0
                flip = c[sd[i][live], 0] != c[i, 0]
                bb = (sd[i][live] == opp[i]) & (src[i][live] == np.flatnonzero(live))
                assert np.all(~flip | bb)


# ---------------------------------------------------------------------------
# P2: mass and x-momentum balance per step

def _perturbed(o, eps=1e-3, seed=3):
    rng = np.random.default_rng(seed)
    drho = eps * rng.uniform(-1, 1, (3, o.nz, o.ny, o.nx))
    u = eps * rng.uniform(-1, 1, (3, 3, o.nz, o.ny, o.nx))
    if o.Q == 9:
        u[:, 2] = 0.0
    o.init_equilibrium(drho, u)


def _post_momentum(o):
    """x-momentum of the post-collision state, per species."""
    gs, _, _ = o.get_state()
    c, _, _ = o.lattice()
    return np.einsum("sik,i->s", gs.reshape(3, o.Q, -1), c[:, 0].astype(float))


@pytest.mark.parametrize("wave", [False, True])
@pytest.mark.parametrize("Q,nx,geo", list(_geometries()))
def test_mass_conserved_per_step(Q, nx, geo, wave):
    o = Oracle(Q, nx, geo, tau=(0.7, 0.6, 1.1), G=(1e-5, 2e-6, 0.0),
               couplings=(0.05, 0.02, 0.1, 0.003, 0.01), phonon_wave=wave)
    _perturbed(o)
    gs0, _, _ = o.get_state()
    m0 = gs0.reshape(3, -1).sum(1)
    for _ in range(5):
        o.step(1)
        gs, _, _ = o.get_state()
        assert np.abs(gs.reshape(3, -1).sum(1) - m0).max() < 1e-15


@pytest.mark.parametrize("wave", [False, True])
@pytest.mark.parametrize("Q", [9, 19])
def test_momentum_balance_without_outer_walls(Q, wave):
    """No void anywhere (periodic in y): the only x-momentum sources are the
    drive on the fluid and the crystal sinks; interface and electron-phonon
    friction cancel pairwise (Eq. 27), specular links carry none.  The same
    holds with the phonons of the damped-wave variant (Sec. 3.4)."""
    rows = [T_SOLID] * 3 + [T_FLUID] * 6 + [T_SOLID] * 2
    G = 3e-5
    o, geo = _mask(Q, 4, rows, tau=(0.7, 0.6, 1.1), G=(G, 0.0, 0.0),
                   couplings=(0.05, 0.02, 0.1, 0.004, 0.01), phonon_wave=wave)
    _perturbed(o)
    n_fluid = (geo.cs_type == T_FLUID).sum() * o.nx
    P0 = _post_momentum(o).sum()
    for _ in range(4):
        f = o.observe()
        solid = np.broadcast_to((geo.cs_type == T_SOLID)[:, :, None], f["u"].shape[2:])
        sinks = 0.004 * f["u"][1, 0][solid].sum() + 0.01 * f["u"][2, 0][solid].sum()
        o.step(1)
        P1 = _post_momentum(o).sum()
        assert abs((P1 - P0) - (G * n_fluid - sinks)) < 1e-15
        P0 = P1


def test_momentum_balance_with_outer_bounceback():
    """With void outside the solid the outer bounce-back links transfer
    2 c_ix g*_opp(i) each; nothing else changes the x-momentum besides the
    drive and the sinks."""
    geo = cross_section("pipe", 17, 15, radius=5, shell=2)
    G = 2e-5
    o = Oracle(19, 3, geo, tau=(0.7, 0.6, 1.1), G=(G, 0, 0),
               couplings=(0.05, 0.02, 0.1, 0.004, 0.01))
    _perturbed(o)
    c, _, opp = o.lattice()
    n_fluid = (geo.cs_type == T_FLUID).sum() * o.nx
    for _ in range(3):
        gs, _, _ = o.get_state()
        gs = gs.reshape(3, 19, -1)
        P0 = np.einsum("sik,i->", gs, c[:, 0].astype(float))
        transfer = 0.0
        for s in range(3):
            src, sd = o.stream_table(s)
            for i in range(19):
                live = src[i] >= 0
                cells = np.flatnonzero(live)
                bb = (sd[i][live] == opp[i]) & (src[i][live] == cells)
                transfer += 2 * c[i, 0] * gs[s, opp[i], cells[bb]].sum()
        f = o.observe()
        solid = np.broadcast_to((geo.cs_type == T_SOLID)[:, :, None], f["u"].shape[2:])
        sinks = 0.004 * f["u"][1, 0][solid].sum() + 0.01 * f["u"][2, 0][solid].sum()
        o.step(1)
        gs1, _, _ = o.get_state()
        P1 = np.einsum("sik,i->", gs1.reshape(3, 19, -1), c[:, 0].astype(float))
        assert abs((P1 - P0) - (G * n_fluid - sinks + transfer)) < 1e-15


# ---------------------------------------------------------------------------
# P3: closed-form special cases

@pytest.mark.parametrize("Q,geo", [
    (9, cross_section("slab", 40, 1, width=32, shell=4)),
    (19, cross_section("pipe", 26, 26, radius=9, shell=3)),
])
def test_free_acceleration(Q, geo):
    """Specular walls and no friction: the fluid accelerates uniformly,
    u_x(n) = G (n + 1/2) / rho0 in every fluid cell."""
    G = 1e-5
    o = Oracle(Q, 3, geo, tau=(0.8, 0.6, 1.0), G=(G, 0, 0))
    o.init_equilibrium()
    fluid = np.broadcast_to((geo.cs_type == T_FLUID)[:, :, None], (geo.nz, geo.ny, 3))
    for n in [0, 1, 7, 50]:
        while o.nstep < n:
            o.step(1)
        u = o.observe()["u"][0]
        assert np.abs(u[0][fluid] - G * (n + 0.5)).max() < 1e-17 + 1e-13 * G * (n + 0.5)
        assert np.abs(u[1:][:, fluid]).max() < 1e-18


@pytest.mark.parametrize("Q,geo", [
    (9, cross_section("slab", 40, 1, width=32, shell=4)),
    (19, cross_section("pipe", 26, 26, radius=9, shell=3)),
])
def test_free_acceleration_observables(Q, geo):
    """The observables of the uniformly accelerating fluid, each from its
    definition: flow rate (1/nx) sum u_x = N_fluid,slice G (n + 1/2),
    wall-row and water means G (n + 1/2), electron and phonon means 0,
    water momentum rho0 N_fluid G (n + 1/2), zero mass deviations, residual
    max |u(n) - u(n-1)| = G, no non-finite value."""
    G, nx, n = 1e-5, 3, 20
    o = Oracle(Q, nx, geo, tau=(0.8, 0.6, 1.0), G=(G, 0, 0))
    o.init_equilibrium()
    o.step(n)
    ob = o.observables()
    n_cs = int((geo.cs_type == T_FLUID).sum())
    u = G * (n + 0.5)
    tol = 1e-12
    assert ob["flow_rate"] == pytest.approx(n_cs * u, rel=tol)
    assert ob["u_wallrow_mean"] == pytest.approx(u, rel=tol)
    assert ob["mean_u"][0] == pytest.approx(u, rel=tol)
    assert abs(ob["mean_u"][1]) < 1e-18 and abs(ob["mean_u"][2]) < 1e-18
    assert ob["momentum"][0] == pytest.approx(n_cs * nx * u, rel=tol)
    assert max(abs(m) for m in ob["mass"]) < 1e-15
    assert ob["residual"] == pytest.approx(G, rel=1e-9)
    assert ob["nonfinite"] == 0 and ob["step"] == n


def test_electron_phonon_crank_nicolson():
    """One uniform solid: delta = u_e - u_p decays by (1 - k/2)/(1 + k/2) per
    step, k = gamma_ep (1/rho_e + 1/rho_p); a phonon sink alone decays u_p by
    (1 - s)/(1 + s), s = gamma_pc / (2 rho_p)."""
    for Q in (9, 19):
        o, geo = _mask(Q, 2, [T_SOLID] * 3, tau=(0.8, 0.6, 1.0), couplings=(0, 0, 0.3, 0, 0))
        u = np.zeros((3, 3, 1, 3, 2))
        u[1, 0] = 0.01
        u[2, 0] = -0.004
        o.init_equilibrium(None, u)
        k = 0.3 * 2.0
        d0 = 0.014
        for n in range(6):
            f = o.observe()
            d = f["u"][1, 0].mean() - f["u"][2, 0].mean()
            expect = d0 * (1 - k / 2) ** n / (1 + k / 2) ** (n + 1)
            assert abs(d - expect) < 1e-15
            tot = f["u"][1, 0].mean() + f["u"][2, 0].mean()
            assert abs(tot - 0.006) < 1e-15
            o.step(1)
        o, geo = _mask(Q, 2, [T_SOLID] * 3, tau=(0.8, 0.6, 1.0), couplings=(0, 0, 0, 0, 0.2))
        o.init_equilibrium(None, u)
        s = 0.1
        for n in range(6):
            up = o.observe()["u"][2, 0].mean()
            assert abs(up - (-0.004) * (1 - s) ** n / (1 + s) ** (n + 1)) < 1e-16
            o.step(1)


def test_lagged_water_electron_pair():
    """A fluid row between solid rows (periodic y, two faces per cell).  With
    the partners coupled through Ubar(n-1) = (u(n-1) + u(n-2))/2 and the Guo
    velocity, D = u_w - u_e obeys
        D(n) = D(n-1) - (k/2) (Dbar(n-2) + Dbar(n-1)),  Dbar(m) = (D(m) + D(m-1))/2,
    k = 2 gamma (1/rho_w + 1/rho_e), with D(-1) = D(-2) = D0 and
    D(0) = (1 - k/2) D0 (derived from rho u(n) = P(n-1) + F(n)/2 and
    P(n) = rho u(n) + F(n)/2).  The pair map is stable for k < 4/3."""
    g = 0.07
    for Q in (9, 19):
        o, geo = _mask(Q, 2, [T_SOLID, T_FLUID], tau=(0.8, 0.6, 1.0), couplings=(g, 0, 0, 0, 0))
        u = np.zeros((3, 3, 1, 2, 2))
        u[0, 0] = 0.02
        u[1, 0] = 0.005
        u[2, 0] = -0.003
        o.init_equilibrium(None, u)
        k = 2 * g * 2.0
        D0 = 0.015
        D = {-2: D0, -1: D0, 0: (1 - k / 2) * D0}
        bar = lambda m: 0.5 * (D[m] + D[m - 1])  # noqa: E731
        for n in range(40):
            if n >= 1:
                D[n] = D[n - 1] - (k / 2) * (bar(n - 2) + bar(n - 1))
            f = o.observe()
            uw = f["u"][0, 0][:, 1].mean()
            ue = f["u"][1, 0][:, 0].mean()
            assert abs((uw - ue) - D[n]) < 1e-15
            assert abs(f["u"][2, 0][:, 0].mean() + 0.003) < 1e-17
            # x-momentum of water + electrons is exchanged, never created
            assert abs(uw + ue - 0.025) < 1e-15
            o.step(1)


def test_lagged_pair_stability_limit():
    """The averaged-lag pair map z^3 - (1 - k/4) z^2 + (k/2) z + k/4 = 0 has
    all roots inside the unit circle exactly for 0 < k < 4/3."""
    rad = lambda k: max(abs(np.roots([1, -(1 - k / 4), k / 2, k / 4])))  # noqa: E731
    assert rad(4 / 3 - 1e-6) < 1 < rad(4 / 3 + 1e-6)
    assert all(rad(k) < 1 for k in np.linspace(0.01, 1.33, 50))


def test_perturbed_start_is_stable_with_strong_couplings():
    """The couplings of the configurations (up to 0.1) leave every mode of a
    perturbed slab and pipe bounded."""
    for Q, geo, nx in [(9, cross_section("slab", 40, 1, width=32, shell=4), 4),
                       (19, cross_section("pipe", 17, 15, radius=5, shell=2), 3)]:
        o = Oracle(Q, nx, geo, tau=(0.55, 0.6, 1.0), G=(1e-5, 0, 0),
                   couplings=(0.1, 0.1, 0.1, 0.0, 0.1))
        _perturbed(o, eps=1e-3, seed=1)
        o.step(1500)
        assert np.abs(o.observe()["u"]).max() < 2e-2


def test_phonon_friction_identity():
    """Sec. 3.4: F_pe + F_pC = -gamma_p u_p with
    gamma_p = gamma_pC + gamma_pe (1 - u_e/u_p)."""
    o, geo = _mask(19, 2, [T_SOLID] * 3, tau=(0.8, 0.6, 1.0), couplings=(0, 0, 0.2, 0, 0.05))
    _perturbed(o, eps=1e-2)
    f = o.observe()
    ue, up, Fp = f["u"][1, 0], f["u"][2, 0], f["F"][2, 0]
    gp = 0.05 + 0.2 * (1 - ue / up)
    assert np.abs(Fp - (-gp * up)).max() < 1e-15


# ---------------------------------------------------------------------------
# Phonons as linear damped waves (Sec. 3.4): the variant whose phonon
# equilibrium is linear in the momentum, g^eq_i = w_i [drho + 3 c_i . rho u].

@pytest.mark.parametrize("Q", [9, 19])
def test_phonon_wave_moments(Q):
    """The linear equilibrium has the moments drho, rho u and cs^2 drho I
    (no convective flux rho u u), its forcing term 0, (1 - omega/2) F and 0;
    water and electrons keep the second-order equilibrium."""
    geo = cross_section("slab", 12, 1, width=4, shell=4) if Q == 9 else \
        cross_section("pipe", 8, 8, radius=2, shell=1)
    o = Oracle(Q, 1, geo, phonon_wave=True)
    ref = Oracle(Q, 1, geo)
    c, w, _ = o.lattice()
    cf = c.astype(float)
    d = 2 if Q == 9 else 3
    I = np.eye(3)
    I[d:, d:] = 0
    rng = np.random.default_rng(11)
    for _ in range(5):
        drho = rng.uniform(-0.05, 0.05)
        rho = 1.0 + drho
        u = rng.uniform(-0.05, 0.05, 3)
        F = rng.uniform(-1e-3, 1e-3, 3)
        if Q == 9:
            u[2] = F[2] = 0.0
        om = rng.uniform(0.6, 1.9)
        eq = np.array([o.geq_species(2, i, drho, u) for i in range(Q)])
        S = np.array([o.guo_species(2, i, om, u, F) for i in range(Q)])
        assert abs(eq.sum() - drho) < 1e-15
        assert np.abs(cf.T @ eq - rho * u).max() < 1e-15
        assert np.abs(np.einsum("i,ia,ib->ab", eq, cf, cf) - drho * CS2 * I).max() < 1e-15
        assert abs(S.sum()) < 1e-16
        assert np.abs(cf.T @ S - (1 - om / 2) * F).max() < 1e-16
        assert np.abs(np.einsum("i,ia,ib->ab", S, cf, cf)).max() < 1e-17
        for s in (0, 1):
            for i in range(Q):
                assert o.geq_species(s, i, drho, u) == ref.geq(i, drho, u)
                assert o.guo_species(s, i, om, u, F) == ref.guo(i, om, u, F)


def _phonon_chain(Q, nx, gamma_pc, tau_p=1.0, wave=True):
    """A periodic chain of solid cells (one cross-section cell, periodic in
    y and z): electrons and phonons only, no interface."""
    geo = cross_section("mask", 1, 1, mask=np.array([[T_SOLID]], np.uint8), periodic_y=True,
                        periodic_z=True)
    return Oracle(Q, nx, geo, tau=(0.8, 0.6, tau_p), couplings=(0, 0, 0, 0, gamma_pc),
                  phonon_wave=wave)


def _damped_mode_fit(a):
    """Decay rate and angular frequency of a sampled damped oscillation
    a(n) = e^{-G n} (A cos w n + B sin w n), from the recurrence
    a(n+1) = 2 e^{-G} cos(w) a(n) - e^{-2G} a(n-1) that it satisfies exactly
    (Prony's method, least squares over all samples)."""
    M = np.stack([a[1:-1], a[:-2]], 1)
    p, *_ = np.linalg.lstsq(M, a[2:], rcond=None)
    r = math.sqrt(-p[1])
    return -math.log(r), math.acos(p[0] / (2 * r))


@pytest.mark.parametrize("Q,gamma_pc,tau_p", [(19, 0.005, 1.0), (19, 0.01, 0.8), (9, 0.005, 1.0)])
def test_phonon_damped_wave_mode(Q, gamma_pc, tau_p):
    """A density mode n_p = eps cos(k x) of the phonon chain follows the damped
    wave equation of Sec. 3.4, d_tt n - cs^2 d_xx n = -gamma_p d_t n (here
    gamma_p = gamma_pC, no electron coupling), plus the BGK viscous damping of
    a longitudinal mode: s^2 + (gamma + 2 nu k^2) s + cs^2 k^2 = 0, i.e. decay
    rate (gamma + 2 nu k^2)/2 and frequency sqrt(cs^2 k^2 - decay^2), with
    nu = cs^2 (tau_p - 1/2) and, for the trapezoidal sink, gamma =
    2 atanh(gamma_pC / 2) (the per-step factor (1 - g/2)/(1 + g/2)).  The
    lattice corrects both at O(k^2) = 6e-4 relative."""
    nx = 256
    o = _phonon_chain(Q, nx, gamma_pc, tau_p)
    k = 2 * math.pi / nx
    x = np.arange(nx)
    drho = np.zeros((3, 1, 1, nx))
    drho[2, 0, 0] = 1e-6 * np.cos(k * x)
    o.init_equilibrium(drho, np.zeros((3, 3, 1, 1, nx)))
    amp = []
    for n in range(2000):
        o.step(1)
        amp.append(o.observe()["drho"][2, 0, 0] @ np.cos(k * x) * 2 / nx)
    decay, freq = _damped_mode_fit(np.array(amp[50:]))
    nu = CS2 * (tau_p - 0.5)
    decay_th = (2 * math.atanh(gamma_pc / 2) + 2 * nu * k * k) / 2
    freq_th = math.sqrt(CS2 * k * k - decay_th ** 2)
    assert decay == pytest.approx(decay_th, rel=1e-4)
    assert freq == pytest.approx(freq_th, rel=3e-4)
    # the sink is what damps the wave: half the rate without it
    assert decay_th > 1.5 * nu * k * k


@pytest.mark.parametrize("wave", [True, False])
def test_phonon_wave_is_linear(wave):
    """With no force the wave variant is a linear scheme: a density mode on
    top of a uniform phonon flow evolves as the two evolve apart (a wave
    equation has no advection term).  The second-order equilibrium advects
    the mode (Doppler shift c_s +- u), so superposition fails by O(1)."""
    nx = 64
    k = 2 * math.pi / nx
    x = np.arange(nx)
    oa, ob, oc = (_phonon_chain(19, nx, 0.0, wave=wave) for _ in range(3))
    drho = np.zeros((3, 1, 1, nx))
    drho[2, 0, 0] = 1e-6 * np.cos(k * x)
    u = np.zeros((3, 3, 1, 1, nx))
    oa.init_equilibrium(drho, u)
    u[2, 0] = 0.05
    ob.init_equilibrium(np.zeros_like(drho), u)
    ga, Ua, U2a = oa.get_state()
    gb, Ub, U2b = ob.get_state()
    oc.set_state(ga + gb, Ua + Ub, U2a + U2b, 0)
    for o in (oa, ob, oc):
        o.step(400)
    ra, rb, rc = (o.observe()["drho"][2, 0, 0] for o in (oa, ob, oc))
    err = np.abs(rc - rb - ra).max() / np.abs(ra).max()
    if wave:
        assert err < 1e-8
    else:
        assert err > 0.1


# ---------------------------------------------------------------------------
# P5-P9: steady slab and pipe

C1 = dict(tau=(0.8, 0.6, 1.0), G=(1e-6, 0, 0), couplings=(0.05, 0.02, 0.1, 0.0, 0.01))


@pytest.mark.slow
def test_magic_tau_bounceback_parabola():
    """Bounce-back walls, no friction: BGK with the Guo source equals TRT
    with Lambda = (tau - 1/2)^2; at Lambda = 3/16 the halfway bounce-back
    parabola is exact: u = G/(2 rho nu) (h^2 - d^2) at every fluid row."""
    G, h = 1e-6, 8.0
    errs = {}
    for tau in (0.5 + math.sqrt(3) / 4, 0.6, 1.5):
        o, geo = _slab(width=16, shell=2, ny=20, tau=(tau, 0.6, 1.0), G=(G, 0, 0),
                       iface_bounceback=True)
        o.init_equilibrium()
        u = _run_to_steady(o, tol=1e-19)[0, 0, 0, :, 0]
        fluid = geo.cs_type[0] == T_FLUID
        prof, _ = slip_poiseuille_slab(G, 1.0, tau, h, 0.0)
        exact = prof(geo.dist[0][fluid])
        errs[tau] = np.abs(u[fluid] - exact).max() / exact.max()
    magic = 0.5 + math.sqrt(3) / 4
    assert errs[magic] < 1e-10
    assert errs[0.6] > 1e-4 and errs[1.5] > 1e-4


def _independent_steady_slab(tau, G, gam, rows, iface_bb=False):
    """Stationary odd-in-c_x equations of the x-invariant D2Q9 slab, solved
    as one dense linear system (independent of the oracle code).

    With a quiescent start the slab keeps rho = rho0 and u_y = 0, and the
    odd part a_i of the post-collision populations with c_x = +1 (E, NE, SE)
    obeys a_i = b_i + omega (3 w_i rho0 u - b_i) + 3 (1 - omega/2) w_i F, with
    b_i its streamed value: a_i of the upstream row, or at a blocked link
    +a_flip(i) (specular) / -a_flip(i) (bounce-back) of the same row,
    flip = c_y reversed.  u = (2 sum_i b_i + F/2) / rho0.  Water:
    F = G - sum_faces [g_we (u_w - u_e) + g_wp (u_w - u_p)]; e/p: trapezoidal
    pair with sinks.
    """
    g_we, g_wp, g_ep, g_ec, g_pc = gam
    ny = len(rows)
    dirs = {"E": (0, 1 / 9), "NE": (1, 1 / 36), "SE": (-1, 1 / 36)}
    flip = {"E": "E", "NE": "SE", "SE": "NE"}
    spec = [(s, y) for y in range(ny) for s in range(3)
            if (rows[y] == T_FLUID) == (s == 0) and rows[y] != 0]
    idx = {}
    for s, y in spec:
        for name in ("E", "NE", "SE", "u", "F"):
            idx[(s, y, name)] = len(idx)
    n = len(idx)
    M = np.zeros((n, n))
    b = np.zeros(n)
    carries = lambda s, y: 0 <= y < ny and rows[y] == (T_FLUID if s == 0 else T_SOLID)  # noqa
    eq = 0

    def streamed(s, y, name):
        cy, _ = dirs[name]
        if carries(s, y - cy):
            return [(1.0, idx[(s, y - cy, name)])]
        void = not (0 <= y - cy < ny) or rows[y - cy] == 0
        sign = -1.0 if (iface_bb or void) else 1.0
        return [(sign, idx[(s, y, flip[name])])]

    for s, y in spec:
        om = 1.0 / tau[s]
        for name, (cy, w) in dirs.items():
            r = eq
            M[r, idx[(s, y, name)]] += 1.0
            for coef, col in streamed(s, y, name):
                M[r, col] -= (1 - om) * coef
            M[r, idx[(s, y, "u")]] -= om * 3 * w
            M[r, idx[(s, y, "F")]] -= 3 * (1 - om / 2) * w
            eq += 1
        r = eq  # rho0 u - F/2 - 2 sum b = 0
        M[r, idx[(s, y, "u")]] += 1.0
        M[r, idx[(s, y, "F")]] -= 0.5
        for name in dirs:
            for coef, col in streamed(s, y, name):
                M[r, col] -= 2 * coef
        eq += 1
        r = eq
        M[r, idx[(s, y, "F")]] += 1.0
        faces = [yy for yy in (y - 1, y + 1) if 0 <= yy < ny and rows[yy] not in (0, rows[y])]
        if s == 0:
            b[r] = G
            for yy in faces:
                M[r, idx[(0, y, "u")]] += g_we + g_wp
                M[r, idx[(1, yy, "u")]] -= g_we
                M[r, idx[(2, yy, "u")]] -= g_wp
        else:
            g_if = g_we if s == 1 else g_wp
            other = 2 if s == 1 else 1
            sink = g_ec if s == 1 else g_pc
            for yy in faces:
                M[r, idx[(s, y, "u")]] += g_if
                M[r, idx[(0, yy, "u")]] -= g_if
            M[r, idx[(s, y, "u")]] += g_ep + sink
            M[r, idx[(other, y, "u")]] -= g_ep
        eq += 1
    assert eq == n
    z = np.linalg.solve(M, b)
    out = np.zeros((3, ny))
    for s, y in spec:
        out[s, y] = z[idx[(s, y, "u")]]
    return out


@pytest.mark.slow
@pytest.mark.parametrize("iface_bb", [False, True])
def test_independent_dense_steady_solve(iface_bb):
    """P8: the time-marched C1 slab reaches the state of the dense solve."""
    rows = [T_SOLID] * 4 + [T_FLUID] * 32 + [T_SOLID] * 4
    o, geo = _slab(iface_bounceback=iface_bb, **C1)
    o.init_equilibrium()
    u = _run_to_steady(o)
    ref = _independent_steady_slab(C1["tau"], 1e-6, C1["couplings"], rows, iface_bb)
    for s in range(3):
        m = ref[s] != 0
        got = u[s, 0, 0, :, 0][m]
        assert np.abs(got - ref[s][m]).max() < 1e-10 * np.abs(ref[0]).max()


@pytest.mark.slow
def test_steady_slab_balance_curvature_and_closed_form():
    """C1 slab at steady state.
    P7: per wall, G H/2 = g_we (u_w,row - u_e,row) + g_wp (u_w,row - u_p,row).
    P6: bulk curvature u_{j+1} - 2 u_j + u_{j-1} = -G/(rho0 nu).
    P9: the fitted profile is the slip Poiseuille closed form; the flow rate
    matches Q(L_s) with the midpoint-sum correction of the cell-centred sum.
    """
    o, geo = _slab(**C1)
    o.init_equilibrium()
    u = _run_to_steady(o)
    uw, ue, up = u[0, 0, 0, :, 0], u[1, 0, 0, :, 0], u[2, 0, 0, :, 0]
    G, H = 1e-6, 32
    bottom = 0.05 * (uw[4] - ue[3]) + 0.02 * (uw[4] - up[3])
    top = 0.05 * (uw[35] - ue[36]) + 0.02 * (uw[35] - up[36])
    assert abs(bottom - G * H / 2) < 1e-12 * G * H
    assert abs(top - G * H / 2) < 1e-12 * G * H
    nu = (0.8 - 0.5) / 3
    curv = uw[15:26] - 2 * uw[14:25] + uw[13:24]
    assert np.abs(curv + G / nu).max() < 1e-9 * G / nu
    obs = o.observables()
    prof, Q = slip_poiseuille_slab(G, 1.0, 0.8, 16.0, obs["slip_length"])
    assert abs(obs["fit_B"] + G / (2 * nu)) < 1e-6 * G / (2 * nu)
    fluid = geo.cs_type[0] == T_FLUID
    d = geo.dist[0][fluid]
    Q_mid = Q + G / (2 * nu) * 2 * 16 / 12.0  # sum_j (h^2 - d_j^2) = 4h^3/3 + h/6
    assert abs(obs["flow_rate"] - Q_mid) < 2e-3 * Q_mid
    assert np.abs(uw[fluid] - prof(d))[4:-4].max() < 1e-6 * uw.max()


@pytest.mark.slow
def test_linear_response_of_slip_length():
    """P9: scaling every coupling by eps, eps * L_s(eps) tends to Navier's
    slip length rho0 nu / (g_we + g_wp): for weak friction the wall-row slip
    carries the whole drive, g_w (u_row - u_solid) = G h, while the solid
    velocities stay bounded (their momentum leaves through the outer walls)."""
    nu = (C1["tau"][0] - 0.5) / 3
    limit = 1.0 * nu / (C1["couplings"][0] + C1["couplings"][1])
    errs = []
    for eps in (1.0, 0.1, 0.01):
        cp = tuple(eps * g for g in C1["couplings"])
        o, geo = _slab(tau=C1["tau"], G=C1["G"], couplings=cp)
        o.init_equilibrium()
        _run_to_steady(o, tol=1e-14 * max(1.0, 1 / eps), chunk=5000, max_steps=2_000_000)
        errs.append(abs(eps * o.observables()["slip_length"] - limit))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.05 * limit
    assert max(e / eps for e, eps in zip(errs, (1.0, 0.1, 0.01))) < 5.0


@pytest.mark.slow
def test_steady_pipe_closed_form():
    """P9 pipe: the fitted curvature and the flow rate follow the slip
    Poiseuille closed form within the staircase error (2%)."""
    geo = cross_section("pipe", 30, 30, radius=11, shell=3)
    tau = 0.7
    G = 1e-6
    o = Oracle(19, 1, geo, tau=(tau, 0.6, 1.0), G=(G, 0, 0),
               couplings=(0.05, 0.02, 0.1, 0.0, 0.01))
    o.init_equilibrium()
    _run_to_steady(o, tol=1e-14, chunk=4000)
    obs = o.observables()
    nu = (tau - 0.5) / 3
    assert abs(obs["fit_B"] + G / (4 * nu)) < 0.02 * G / (4 * nu)
    _, Q = slip_poiseuille_pipe(G, 1.0, tau, geo.d_wall, obs["slip_length"])
    assert abs(obs["flow_rate"] - Q) < 0.02 * Q
    # P7 for the pipe: at steady state the drive on the water of a slice
    # equals the interface friction summed over its fluid/solid faces
    # (specular faces carry no momentum), exactly.
    u = o.observe()["u"]
    uw, ue, up = u[0][0][..., 0], u[1][0][..., 0], u[2][0][..., 0]
    t = geo.cs_type
    g_we, g_wp = 0.05, 0.02
    friction = 0.0
    for z, y in zip(*np.nonzero(t == T_FLUID)):
        for dz, dy in ((0, 1), (0, -1), (1, 0), (-1, 0)):
            zz, yy = z + dz, y + dy
            if 0 <= zz < geo.nz and 0 <= yy < geo.ny and t[zz, yy] == T_SOLID:
                friction += g_we * (uw[z, y] - ue[zz, yy]) + g_wp * (uw[z, y] - up[zz, yy])
    drive = G * int((t == T_FLUID).sum())
    assert abs(friction - drive) < 1e-9 * drive


# ---------------------------------------------------------------------------
# P10: D3Q19 z-invariant slab = D2Q9 slab; eight-fold pipe symmetry

def test_d3q19_slab_equals_d2q9_slab():
    o2, _ = _slab(Q=9, nx=3, **C1)
    geo3 = cross_section("slab", 40, 1, width=32, shell=4)
    o3 = Oracle(19, 3, geo3, **C1)
    o2.init_equilibrium()
    o3.init_equilibrium()
    for _ in range(6):
        o2.step(100)
        o3.step(100)
        u2 = o2.observe()["u"][:, 0]
        u3 = o3.observe()["u"][:, 0]
        assert np.abs(u2 - u3).max() < 1e-12 * np.abs(u2).max()


def test_pipe_eightfold_symmetry():
    geo = cross_section("pipe", 24, 24, radius=8, shell=3)
    o = Oracle(19, 2, geo, tau=(0.7, 0.6, 1.0), G=(1e-5, 0, 0),
               couplings=(0.05, 0.02, 0.1, 0.0, 0.01))
    o.init_equilibrium()
    o.step(300)
    f = o.observe()
    for s in range(3):
        ux = f["u"][s, 0][:, :, 0]  # (z, y)
        scale = np.abs(ux).max()
        assert scale > 0
        for img in (ux.T, ux[::-1, :], ux[:, ::-1]):
            assert np.abs(ux - img).max() < 1e-12 * scale
        uy, uz = f["u"][s, 1][:, :, 0], f["u"][s, 2][:, :, 0]
        assert np.abs(uy - uz.T).max() < 1e-12 * scale


# ---------------------------------------------------------------------------
# Negative quantum friction (Sec. 2: the couplings may "go both ways"):
# a negative water-electron coupling inside the stability bound.

NEG = dict(tau=(0.8, 0.6, 1.0), G=(1e-6, 0, 0), couplings=(-0.02, 0.05, 0.1, 0.0, 0.01))


def test_negative_friction_steady_slab():
    """With g_we < 0 the steady slab still balances the drive at each wall
    (P7: G H/2 = g_we (u_w - u_e) + g_wp (u_w - u_p), here with one term of
    each sign), and equals the independent dense steady solve (P8)."""
    rows = [T_SOLID] * 4 + [T_FLUID] * 32 + [T_SOLID] * 4
    o, geo = _slab(**NEG)
    o.init_equilibrium()
    u = _run_to_steady(o)
    uw, ue, up = u[0, 0, 0, :, 0], u[1, 0, 0, :, 0], u[2, 0, 0, :, 0]
    G, H = 1e-6, 32
    bottom = -0.02 * (uw[4] - ue[3]) + 0.05 * (uw[4] - up[3])
    assert abs(bottom - G * H / 2) < 1e-12 * G * H
    assert -0.02 * (uw[4] - ue[3]) < 0  # the electron term pushes the water
    ref = _independent_steady_slab(NEG["tau"], 1e-6, NEG["couplings"], rows)
    for s in range(3):
        m = ref[s] != 0
        assert np.abs(u[s, 0, 0, :, 0][m] - ref[s][m]).max() < 1e-10 * np.abs(ref[0]).max()


# ---------------------------------------------------------------------------
# Thermal fluctuations (Eq. 6, Eq. 17): the generator, exact conservation,
# and equipartition of the fluctuating lattice fluid.

def test_philox_known_answer_vectors():
    """The oracle's Philox-4x32-10 reproduces the generator's published
    known-answer vectors (Salmon et al., SC 2011; fixture
    tests/golden/philox4x32_10_kat.txt): a swapped output word, a wrong
    multiplier or Weyl constant, or a wrong round count changes every word."""
    from oracle.oracle import philox4x32_10

    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        got = [int(x) for x in philox4x32_10(v[0:4], v[4:6])]
        assert got == v[6:10], (r, [f"{x:08x}" for x in got])


def test_philox_generator_statistics():
    """Philox-4x32-10 words are uniform, uncorrelated between neighbouring
    counters and words, distinct over a sample of counters (the map is a
    bijection of the counter), and change about half their bits when one key
    bit flips."""
    from oracle.oracle import philox4x32_10

    n = 4096
    out = np.array([philox4x32_10([c, 7, 0, k], [0x1234, 0x9abc]) for c in range(n // 4) for k in range(4)],
                   np.uint64).ravel()
    u = (out.astype(np.float64) + 0.5) / 2.0 ** 32
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / u.size)
    assert abs(u.var() - 1 / 12) < 0.05 / 12
    hist, _ = np.histogram(u, bins=64, range=(0, 1))
    chi2 = ((hist - u.size / 64) ** 2 / (u.size / 64)).sum()
    assert chi2 < 63 + 5 * math.sqrt(2 * 63)
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 4 / math.sqrt(u.size)
    assert len(np.unique(out)) == out.size
    a = np.array([philox4x32_10([c, 0, 0, 0], [1, 2]) for c in range(256)], np.uint32)
    b = np.array([philox4x32_10([c, 0, 0, 0], [1 ^ 8, 2]) for c in range(256)], np.uint32)
    flips = np.unpackbits((a ^ b).view(np.uint8)).mean()
    assert abs(flips - 0.5) < 0.03


def test_thermal_noise_conserves_mass_and_momentum():
    """The noise is projected off mass and momentum: with no drive and no
    coupling the water's total mass and x-momentum stay at zero to rounding
    while the populations fluctuate."""
    geo = cross_section("slab", 24, 1, width=16, shell=4)
    o = Oracle(9, 16, geo, tau=(0.8, 0.6, 1.0), G=(0, 0, 0), couplings=(0, 0, 0, 0, 0))
    o.init_equilibrium()
    o.set_fluctuations(1e-5, 99)
    o.step(50)
    f = o.observe()
    fluid = np.broadcast_to((geo.cs_type == 1)[..., None], f["drho"][0].shape)
    d = f["drho"][0][fluid]
    jx = ((1.0 + f["drho"][0]) * f["u"][0][0])[fluid]
    assert np.abs(d).max() > 1e-4  # fluctuating
    assert abs(d.sum()) < 1e-12 and abs(jx.sum()) < 1e-12


@pytest.mark.parametrize("Q,tau", [(9, 0.8), (9, 1.0), (19, 0.8)])
def test_equipartition(Q, tau):
    """Fluctuation-dissipation of the lattice fluid: at rest with thermal
    noise every velocity component of a fluid cell has rho0 <u_a^2> = kT and
    the density <drho^2> = rho0 kT / cs^2 (slab with specular walls, isolated
    water).  Tolerance: 3% (several thousand effectively independent
    samples)."""
    nz = 1 if Q == 9 else 4
    geo = cross_section("slab", 24, nz, width=16, shell=4)
    o = Oracle(Q, 32, geo, tau=(tau, 0.6, 1.0), G=(0, 0, 0), couplings=(0, 0, 0, 0, 0))
    o.init_equilibrium()
    kT = 1e-5
    o.set_fluctuations(kT, 2024)
    o.step(500)
    fluid = geo.cs_type == 1
    acc, n = np.zeros(4), 0
    for _ in range(200 if Q == 9 else 60):
        o.step(5)
        f = o.observe()
        m = np.broadcast_to(fluid[..., None], f["drho"][0].shape)
        u = f["u"][0]
        acc += [np.mean(u[0][m] ** 2), np.mean(u[1][m] ** 2), np.mean(u[2][m] ** 2),
                np.mean(f["drho"][0][m] ** 2)]
        n += 1
    acc /= n
    assert acc[0] == pytest.approx(kT, rel=0.03)
    assert acc[1] == pytest.approx(kT, rel=0.03)
    if Q == 19:
        assert acc[2] == pytest.approx(kT, rel=0.03)
    assert acc[3] == pytest.approx(3 * kT, rel=0.03)
