"""Pins of the oracle's bead forces, integrator, noise and coupling weights.

* Every conservative force is minus the gradient of its energy (central
  finite differences on the oracle's energies), and the two-bead WCA force has
  the closed form 24 eps (2 (s/r)^12 - (s/r)^6) / r.
* Internal forces sum to zero (Newton's third law); the angular term vanishes
  for a straight chain.
* With no friction, noise or field the multiple-time-step cycle is plain
  velocity Verlet with dt = 1/(M M^b): energy is conserved to O(dt^2).
* A free bead in a fluid at rest loses velocity as exp(-gamma t) to first
  order in the MD step (Sec. II, Eq. 12).
* The Philox4x32-10 normals have zero mean, unit variance and no correlation
  between beads, components, substeps and steps; a bead's velocity variance
  reaches kT (Sec. II, Eq. 15, fluctuation-dissipation).
* Trilinear weights: sum to one, reproduce linear fields, give the node value
  at a node, vanish on solid corners, and wrap periodically.
"""
import numpy as np
import pytest

from paper_0711_2665_gb300 import inputs


def _sim(orc, n, solid=None, dims=(16, 12, 12), **kw):
    p = dict(nx=dims[0], ny=dims[1], nz=dims[2], tau=0.8, n_beads=n, k_bond=100.0, r0=1.0,
             kappa_bend=0.7, lj_sigma=1.0, lj_eps=1.0, wall_sigma=1.0, wall_eps=1.0,
             E=0.0, gamma=0.1, kT=0.0, md_outer=5, md_inner=20, seed=5, wall_x=-1, pore_h=3)
    p.update(kw)
    return orc.OracleSim(p, solid)


def _fd_forces(sim, r, h=1e-6):
    F = np.zeros_like(r)
    for i in range(r.shape[0]):
        for a in range(3):
            rp, rm = r.copy(), r.copy()
            rp[i, a] += h
            rm[i, a] -= h
            F[i, a] = -(sim.fast_energies(rp).sum() - sim.fast_energies(rm).sum()) / (2 * h)
    return F


def _crumpled_chain(n, seed, spacing=0.97):
    """A compact chain with bond lengths near 1, random angles and several
    non-bonded pairs inside the WCA range."""
    rng = np.random.default_rng(seed)
    r = np.zeros((n, 3))
    r[0] = [6.3, 6.1, 5.9]
    for i in range(1, n):
        while True:
            d = rng.normal(size=3)
            d *= spacing * (1 + 0.05 * rng.normal()) / np.linalg.norm(d)
            p = r[i - 1] + d
            if i < 2 or np.min(np.linalg.norm(r[:i - 1] - p, axis=1)) > 0.9:
                break
        r[i] = p
    return r


def test_forces_are_minus_energy_gradient(orc):
    r = _crumpled_chain(12, 1)
    sim = _sim(orc, 12)
    e = sim.fast_energies(r)
    assert e[0] > 0 and e[1] > 0 and e[2] > 0  # bonds, bending, WCA all active
    F = sim.fast_forces(r)
    Ffd = _fd_forces(sim, r)
    assert np.allclose(F, Ffd, rtol=1e-6, atol=1e-6 * np.abs(F).max())
    assert np.allclose(F.sum(0), 0.0, atol=1e-10 * np.abs(F).max())


def test_wall_force_is_minus_energy_gradient(orc):
    solid = inputs.pore_wall_mask(16, 12, 12, 7, 3)
    r = np.array([[6.2, 3.3, 4.1], [6.5, 4.0, 4.6], [7.5, 3.8, 5.2], [7.9, 5.0, 5.1]])
    sim = _sim(orc, 4, solid=solid, k_bond=0.0, kappa_bend=0.0, lj_eps=0.0)
    e = sim.fast_energies(r)
    assert e[3] > 0
    F = sim.fast_forces(r)
    assert np.allclose(F, _fd_forces(sim, r), rtol=1e-6, atol=1e-7 * np.abs(F).max())


def test_two_bead_wca_closed_form(orc):
    sim = _sim(orc, 3, k_bond=0.0, kappa_bend=0.0)
    for d in (0.9, 1.0, 1.05, 1.12, 1.13):
        r = np.array([[4.0, 4.0, 4.0], [8.0, 8.0, 8.0], [4.0 + d, 4.0, 4.0]])  # beads 0 and 2
        F = sim.fast_forces(r)
        rc = 2 ** (1 / 6)
        expect = 24 * (2 * d ** -12 - d ** -6) / d if d < rc else 0.0
        assert F[2, 0] == pytest.approx(expect, rel=1e-13, abs=1e-13)
        assert F[0, 0] == pytest.approx(-expect, rel=1e-13, abs=1e-13)
        e = sim.fast_energies(r)[2]
        assert e == pytest.approx(4 * (d ** -12 - d ** -6) + 1 if d < rc else 0.0, abs=1e-13)


def test_bonded_neighbours_do_not_feel_wca(orc):
    sim = _sim(orc, 2, k_bond=0.0, kappa_bend=0.0)
    r = np.array([[4.0, 4.0, 4.0], [4.9, 4.0, 4.0]])
    assert np.allclose(sim.fast_forces(r), 0.0)


def test_wca_uses_minimum_image(orc):
    sim = _sim(orc, 3, k_bond=0.0, kappa_bend=0.0)
    r = np.array([[0.3, 4.0, 4.0], [6.0, 6.0, 6.0], [15.3 + 16.0, 4.0, 4.0]])  # 1.0 apart through x
    F = sim.fast_forces(r)
    assert F[0, 0] == pytest.approx(24.0, rel=1e-12)
    assert F[2, 0] == pytest.approx(-24.0, rel=1e-12)


def test_bending_straight_chain_and_small_angle(orc):
    kappa = 0.7
    sim = _sim(orc, 3, k_bond=0.0, lj_eps=0.0, kappa_bend=kappa)
    r = np.array([[3.0, 3.0, 3.0], [4.0, 3.0, 3.0], [5.0, 3.0, 3.0]])
    assert sim.fast_energies(r)[1] == 0.0
    assert np.allclose(sim.fast_forces(r), 0.0, atol=1e-14)
    # small angle: transverse displacement eps of the end bead -> phi ~ eps,
    # restoring force on it ~ -kappa phi (lever arm 1)
    eps = 1e-4
    r[2, 1] += eps
    F = sim.fast_forces(r)
    phi = np.arctan2(eps, 1.0)
    assert sim.fast_energies(r)[1] == pytest.approx(0.5 * kappa * phi ** 2, rel=1e-9)
    assert F[2, 1] == pytest.approx(-kappa * phi, rel=1e-6)


def test_bond_force_closed_form(orc):
    sim = _sim(orc, 2, kappa_bend=0.0, lj_eps=0.0, k_bond=100.0, r0=1.0)
    r = np.array([[3.0, 3.0, 3.0], [3.0, 4.2, 3.0]])
    F = sim.fast_forces(r)
    assert F[1, 1] == pytest.approx(-100.0 * 0.2, rel=1e-13)
    assert F[0, 1] == pytest.approx(100.0 * 0.2, rel=1e-13)


def test_inner_cycle_is_velocity_verlet_and_conserves_energy(orc):
    """gamma = kT = E = 0: beads decouple from the fluid; one LB step is
    M * M^b velocity-Verlet steps of dt = 1/(M M^b) on the conservative
    forces.  Check against a plain Verlet loop driven by the oracle's force
    routine, then check energy conservation over many steps."""
    n = 10
    r0 = _crumpled_chain(n, 4, spacing=1.02)
    rng = np.random.default_rng(2)
    v0 = 0.2 * rng.standard_normal((n, 3))
    sim = _sim(orc, n, gamma=0.0)
    sim.set_beads(r0, v0)
    sim.step(1)
    r1, v1 = sim.get_beads()
    dt = 1.0 / 100
    r, v = r0.copy(), v0.copy()
    for _ in range(100):
        v += 0.5 * dt * sim.fast_forces(r)
        r += dt * v
        v += 0.5 * dt * sim.fast_forces(r)
    assert np.allclose(r1, r, atol=1e-12) and np.allclose(v1, v, atol=1e-12)

    def energy(rr, vv):
        return sim.fast_energies(rr).sum() + 0.5 * (vv * vv).sum()

    e0 = energy(r1, v1)
    es = []
    for _ in range(40):
        sim.step(1)
        es.append(energy(*sim.get_beads()))
    drift = np.max(np.abs(np.array(es) - e0))
    assert drift < 2e-3 * e0


def test_friction_decay_of_a_free_bead(orc):
    """One bead, fluid at rest, no other forces: over one LB step the velocity
    decays as exp(-gamma) up to the first-order splitting error O(gamma^2 dt)."""
    gamma = 0.1
    sim = _sim(orc, 1, dims=(24, 24, 24), gamma=gamma)
    v0 = np.array([[0.01, 0.0, 0.0]])
    sim.set_beads(np.array([[11.5, 12.2, 12.7]]), v0)
    sim.step(1)
    _, v1 = sim.get_beads()
    assert abs(v1[0, 0] / v0[0, 0] - np.exp(-gamma)) < 5e-4
    up, J = sim.last_coupling()
    assert np.allclose(up, 0.0)
    assert J[0, 0] == pytest.approx(v1[0, 0] - v0[0, 0], rel=1e-12)


def test_philox_normals_statistics(orc):
    """10^6 normals over beads x substeps x steps: mean 0 and variance 1
    within 5 sigma; no correlation between components, beads or steps."""
    zs = []
    for step in range(20):
        for sub in range(5):
            zs.append(orc.gauss3_batch(7, 3, 3334, step, sub))
    z = np.stack(zs)  # (100, 3334, 3)
    flat = z.reshape(-1)
    n = flat.size
    assert abs(flat.mean()) < 5 / np.sqrt(n)
    assert abs(flat.var() - 1) < 5 * np.sqrt(2 / n)
    # kurtosis of a normal is 3
    assert abs(np.mean(flat ** 4) - 3) < 5 * np.sqrt(96 / n)
    tol = 5 / np.sqrt(z.shape[0] * z.shape[1])
    for a, b in ((0, 1), (0, 2), (1, 2)):
        assert abs(np.mean(z[..., a] * z[..., b])) < tol
    assert abs(np.mean(z[:, :-1, 0] * z[:, 1:, 0])) < tol          # neighbouring beads
    assert abs(np.mean(z[:-5, :, 0] * z[5:, :, 0])) < tol          # consecutive steps
    assert abs(np.mean(z[:-1, :, 1] * z[1:, :, 1])) < tol          # consecutive substeps
    # different realizations and seeds give different streams
    assert not np.allclose(orc.gauss3_batch(7, 4, 10, 0, 0), orc.gauss3_batch(7, 3, 10, 0, 0))
    assert not np.allclose(orc.gauss3_batch(8, 3, 10, 0, 0), orc.gauss3_batch(7, 3, 10, 0, 0))


def test_philox_uniform_words(orc):
    """The 32-bit words are uniform: chi^2 over 64 bins of the top 6 bits."""
    words = np.array([orc.philox4x32_10([i, 17, 3, 0], [99, 1]) for i in range(20000)]).reshape(-1)
    hist = np.bincount(words >> 26, minlength=64)
    expect = words.size / 64
    chi2 = ((hist - expect) ** 2 / expect).sum()
    assert chi2 < 63 + 5 * np.sqrt(2 * 63)


def test_bead_velocity_variance_reaches_kT(orc):
    """Sec. II, Eq. 15: noise of variance 2 gamma kT / m per unit time balances
    the friction, so <v_a^2> -> kT.  Free beads (no bonds, bending or overlap)
    in a large box; the fluid heats up by a negligible amount."""
    kT = 1e-4
    n = 64
    g = np.stack(np.meshgrid(np.arange(4), np.arange(4), np.arange(4), indexing="ij"), -1)
    r = 3.0 + 4.0 * g.reshape(-1, 3).astype(float) + 0.3
    sim = _sim(orc, n, dims=(16, 16, 16), k_bond=0.0, kappa_bend=0.0, gamma=0.5, kT=kT, seed=11)
    sim.set_beads(r)
    sim.step(20)
    acc = []
    for _ in range(60):
        sim.step(1)
        acc.append(sim.get_beads()[1])
    v2 = np.mean(np.array(acc) ** 2)
    # samples are correlated over ~1/gamma = 2 steps -> ~ 64*3*60/2 independent
    assert abs(v2 / kT - 1) < 0.1


def test_trilinear_weights(orc):
    solid = inputs.pore_wall_mask(8, 8, 8, 5, 2)
    sim = _sim(orc, 1, solid=solid, dims=(8, 8, 8))
    rng = np.random.default_rng(0)
    # away from walls: reproduces a linear field, weights sum to 1
    for _ in range(20):
        r = np.array([rng.uniform(1, 3.9), rng.uniform(0, 8), rng.uniform(0, 8)])
        nodes, w, nf = sim.interp_weights(r)
        assert nf == 8 and abs(w.sum() - 1) < 1e-15
        xs = np.array([[n % 8, (n // 8) % 8, n // 64] for n in nodes], dtype=float)
        # unwrap node coordinates next to the bead for the linear-field check
        xs = xs + 8 * np.round((r - xs) / 8)
        lin = lambda q: 0.3 + 1.7 * q[..., 0] - 0.2 * q[..., 1] + 0.9 * q[..., 2]
        assert abs(w @ lin(xs) - lin(r)) < 1e-12
    # at a node: weight 1 on that node
    nodes, w, _ = sim.interp_weights(np.array([2.0, 3.0, 6.0]))
    assert w.max() == 1.0 and nodes[np.argmax(w)] == 2 + 8 * (3 + 8 * 6)
    # next to the wall: solid corners get 0, the rest renormalised
    nodes, w, nf = sim.interp_weights(np.array([4.5, 0.5, 0.5]))
    assert nf == 4 and abs(w.sum() - 1) < 1e-15
    assert np.all(w[[1, 3, 5, 7]] == 0) and np.allclose(w[[0, 2, 4, 6]], 0.25)
    # periodic wrap: x = 7.5 mixes nodes 7 and 0
    nodes, w, _ = sim.interp_weights(np.array([7.5, 2.0, 2.0]))
    assert set((nodes[w > 0] % 8).tolist()) == {7, 0}
    nodes2, w2, _ = sim.interp_weights(np.array([7.5 - 8.0, 2.0, 2.0]))
    assert np.array_equal(nodes, nodes2) and np.allclose(w, w2)


def test_pore_channel_region(orc):
    """The field acts inside |x - wall_x| <= 3/2 and within the pore's cross
    section padded by half a site (h = 3 pore at y, z in {5, 6, 7} for n = 12)."""
    sim = _sim(orc, 5, dims=(16, 12, 12), wall_x=8, pore_h=3, E=0.1, k_bond=0.0,
               kappa_bend=0.0)
    r = np.array([[8.0, 6.0, 6.0], [9.5, 6.0, 6.0], [9.6, 6.0, 6.0], [8.0, 7.5, 4.5],
                  [8.0, 7.6, 6.0]])
    F = sim.field_forces(r)
    assert F[:, 0].tolist() == [0.1, 0.1, 0.0, 0.1, 0.0]
    assert np.all(F[:, 1:] == 0)
