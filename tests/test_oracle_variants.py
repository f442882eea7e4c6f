"""Pins of the oracle's variants of the coupled step.

Nearest-grid-point coupling (the paper's own scheme, Sec. II): the weights are
one at the lattice site nearest to the bead (brute force over the cell's
corners, periodic) and zero elsewhere, or zero everywhere when that site is
solid; fluid + bead momentum stays constant; the adjoint matches central
differences with the field events held.

Stochastic position Verlet (Sec. II, Eq. SPValgo, nested): for a free bead in
a held fluid velocity U the velocity relaxes as U + (v0 - U) exp(-gamma t)
exactly at any step size; the stationary velocity variance is kT exactly even
at gamma h = 1, where the explicit-friction Verlet cycle is visibly off; without
friction and noise the cycle is position Verlet, time-reversible to rounding;
fluid + bead momentum stays constant, and without friction the impulse the
fluid gives (v' - v - h F) vanishes.
"""
import numpy as np
import pytest

from paper_0711_2665_gb300 import inputs

BOX = (12, 10, 10)


def _sim(orc, solid=None, **kw):
    p = dict(nx=BOX[0], ny=BOX[1], nz=BOX[2], tau=0.8, n_beads=6, k_bond=100.0, r0=1.0, kappa_bend=1e-3,
             lj_sigma=1.0, lj_eps=1.0, wall_sigma=1.0, wall_eps=1.0, E=0.0, gamma=0.1,
             kT=1e-4, md_outer=5, md_inner=20, seed=123, wall_x=-1, pore_h=3)
    p.update(kw)
    return orc.OracleSim(p, solid), p


def _total_momentum(o):
    return np.array([o["p_fluid_x"] + o["p_beads_x"], o["p_fluid_y"] + o["p_beads_y"],
                     o["p_fluid_z"] + o["p_beads_z"]])


def test_nearest_grid_point_weights(orc):
    solid = inputs.pore_wall_mask(*BOX, 6, 3)
    sim, p = _sim(orc, solid=solid, interp=1, wall_x=6)
    rng = np.random.default_rng(0)
    box = np.array(BOX, float)
    flat = solid.reshape(-1)
    for _ in range(400):
        r = rng.uniform(-3.0, 15.0, size=3)
        nodes, w, _ = sim.interp_weights(r)
        rw = r - box * np.floor(r / box)
        c0 = np.floor(rw).astype(int)
        best, bestd = None, 1e9
        for k in range(8):
            c = c0 + np.array([k & 1, (k >> 1) & 1, k >> 2])
            d = np.linalg.norm(rw - c)
            if d < bestd:
                best, bestd = k, d
        cn = (c0 + np.array([best & 1, (best >> 1) & 1, best >> 2])) % np.array(BOX)
        site = cn[0] + BOX[0] * (cn[1] + BOX[1] * cn[2])
        if flat[site]:
            assert np.all(w == 0.0)
        else:
            assert w[best] == 1.0 and np.count_nonzero(w) == 1 and nodes[best] == site


@pytest.mark.parametrize("variant", [dict(interp=1), dict(integrator=1), dict(interp=1, integrator=1)])
def test_variants_conserve_momentum(orc, variant):
    sim, p = _sim(orc, **variant)
    rng = np.random.default_rng(3)
    r = inputs.chain_walk(6, BOX, -1, np.zeros(BOX[::-1], np.uint8), 9)
    sim.set_beads(r, 0.05 * rng.standard_normal((6, 3)))
    P0 = _total_momentum(sim.observables())
    sim.step(30)
    P1 = _total_momentum(sim.observables())
    assert np.all(np.abs(P0) > 1e-3)
    assert np.allclose(P1, P0, atol=1e-13)
    assert abs(sim.observables()["p_fluid_x"]) > 1e-3


def test_nearest_grid_point_adjoint_matches_held_event_differences(orc):
    dims, wall, K, h = (20, 12, 12), 10, 6, 1e-4
    solid = inputs.pore_wall_mask(*dims, wall, 3)
    P = dict(nx=dims[0], ny=dims[1], nz=dims[2], tau=0.8, wall_x=wall, pore_h=3, n_beads=6,
             kappa_bend=1e-3, E=0.1, gamma=0.1, kT=1e-4, seed=7, interp=1)
    r0 = inputs.chain_walk(6, dims, wall, solid, 3)
    r0[:, 0] += 0.3
    r0[:, 1:] += 0.137
    g = orc.adjoint(P, solid, r0, K)
    s = orc.OracleSim(P, solid)
    s.set_beads(r0)
    trace = np.zeros(K * 10 * 6, np.int32)
    s.channel_trace(1, trace)
    s.step(K)

    def loss(params, r):
        q = orc.OracleSim(params, solid)
        q.set_beads(r)
        q.channel_trace(2, trace)
        q.step(K)
        return q.get_beads()[0][:, 0].mean() - r[:, 0].mean(), q.event_counts()[1]

    for name in ("gamma", "E"):
        Pp, Pm = dict(P), dict(P)
        Pp[name] += h
        Pm[name] -= h
        (lp, ep), (lm, em) = loss(Pp, r0), loss(Pm, r0)
        assert ep == em
        assert g["d" + name] == pytest.approx((lp - lm) / (2 * h), rel=1e-4), name
    scale = np.abs(g["dr0"]).max()
    checked = 0
    for i, a in ((0, 0), (1, 2), (4, 1), (5, 0)):
        rp, rm = r0.copy(), r0.copy()
        rp[i, a] += h
        rm[i, a] -= h
        (lp, ep), (lm, em) = loss(P, rp), loss(P, rm)
        if ep != em:  # a bead crossed a mid-plane between the cells' nodes
            continue
        checked += 1
        assert abs(g["dr0"][i, a] - (lp - lm) / (2 * h)) <= 1e-3 * scale + 1e-3 * abs(lp - lm) / (2 * h)
    assert checked >= 3


def _free_beads(orc, n, **kw):
    """n beads with no conservative forces (no bonds, angles or WCA)."""
    p = dict(n_beads=n, k_bond=0.0, kappa_bend=0.0, lj_eps=0.0, wall_sigma=1.0, integrator=1)
    p.update(kw)
    return _sim(orc, **p)


def test_spv_exact_relaxation(orc):
    gamma, M, Mb, n = 0.7, 2, 3, 9
    sim, p = _free_beads(orc, 1, gamma=gamma, kT=0.0, md_outer=M, md_inner=Mb)
    U = np.array([[0.02, -0.01, 0.005]])
    v0 = np.array([[0.1, 0.2, -0.3]])
    sim.set_beads(np.array([[5.3, 4.1, 3.7]]), v0)
    sim.md_only(U, n)
    _, v = sim.get_beads()
    expect = U + (v0 - U) * np.exp(-gamma * n)
    assert np.allclose(v, expect, rtol=0, atol=1e-14)


@pytest.mark.parametrize("integrator,exact", [(1, True), (0, False)])
def test_spv_stationary_variance_at_large_steps(orc, integrator, exact):
    """gamma h = 1 (M = M^b = 1): the exact Ornstein-Uhlenbeck update keeps
    the variance at kT; the explicit friction of the Verlet cycle does not."""
    kT, n_beads = 1e-4, 3000
    sim, p = _free_beads(orc, n_beads, gamma=1.0, kT=kT, md_outer=1, md_inner=1, integrator=integrator)
    rng = np.random.default_rng(1)
    sim.set_beads(rng.uniform(0, 10, size=(n_beads, 3)), np.sqrt(kT) * rng.standard_normal((n_beads, 3)))
    U = np.zeros((n_beads, 3))
    acc = []
    for k in range(60):
        sim.md_only(U, 1)
        if k >= 10:
            acc.append(np.mean(sim.get_beads()[1] ** 2))
    ratio = np.mean(acc) / kT
    if exact:
        assert abs(ratio - 1.0) < 0.02, ratio
    else:
        assert abs(ratio - 1.0) > 0.05, ratio


def test_spv_without_friction_is_time_reversible(orc):
    sim, p = _sim(orc, integrator=1, gamma=0.0, kT=0.0, kappa_bend=0.5)
    r = inputs.chain_walk(6, BOX, -1, np.zeros(BOX[::-1], np.uint8), 9)
    rng = np.random.default_rng(2)
    v0 = 0.3 * rng.standard_normal((6, 3))
    sim.set_beads(r, v0)
    U = np.zeros((6, 3))
    e0 = sim.fast_energies(r).sum() + 0.5 * np.sum(v0 ** 2)
    sim.md_only(U, 4)
    r1, v1 = sim.get_beads()
    # without friction the fluid gives nothing: J = v' - v - h F vanishes
    assert np.abs(sim.last_coupling()[1]).max() < 1e-14
    e1 = sim.fast_energies(r1).sum() + 0.5 * np.sum(v1 ** 2)
    assert abs(e1 - e0) < 1e-3 * e0
    sim.set_beads(r1, -v1)
    sim.md_only(U, 4)
    r2, v2 = sim.get_beads()
    assert np.allclose(r2, r, atol=1e-10) and np.allclose(v2, -v0, atol=1e-9)
