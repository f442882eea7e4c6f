"""Pins of the oracle's lattice tables, equilibrium, source and collision.

Each check compares the oracle with a property that the mathematics fixes
(isotropy of the D3Q19 weights, closed-form moments of the equilibrium,
the exact moments the source must have by Sec. II, Eqs. 8-9) rather than with
a retyped copy of its own formulas.
"""
import itertools

import numpy as np
import pytest


def test_d3q19_velocity_set(orc):
    c, w, opp = orc.tables()
    # 19 distinct velocities: rest, 6 first neighbours, 12 second neighbours
    assert len({tuple(v) for v in c}) == 19
    n2 = (c * c).sum(1)
    assert sorted(n2.tolist()) == [0] + [1] * 6 + [2] * 12
    assert np.all(np.abs(c) <= 1)
    # opposite table
    for i in range(19):
        assert np.array_equal(c[opp[i]], -c[i])
        assert opp[opp[i]] == i


def test_d3q19_isotropy(orc):
    """sum w = 1, sum w c = 0, sum w c_a c_b = I/3, third moment 0, fourth
    moment = (d_ab d_cd + d_ac d_bd + d_ad d_bc)/9 -- the lattice conditions
    that give Navier-Stokes with c_s^2 = 1/3."""
    c, w, _ = orc.tables()
    c = c.astype(float)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose((w[:, None] * c).sum(0), 0.0, atol=1e-16)
    m2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(m2, np.eye(3) / 3.0, atol=1e-15)
    m3 = np.einsum("i,ia,ib,ic->abc", w, c, c, c)
    assert np.allclose(m3, 0.0, atol=1e-16)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(m4, iso, atol=1e-15)


@pytest.mark.parametrize("rho,u", [(1.0, (0.0, 0.0, 0.0)), (1.02, (0.05, -0.03, 0.01)),
                                   (0.97, (-0.1, 0.08, 0.12)), (2.5, (0.0, 0.0, -0.2))])
def test_equilibrium_moments(orc, rho, u):
    """sum feq = rho, sum feq c = rho u, sum feq c c = rho/3 I + rho u u."""
    c, _, _ = orc.tables()
    c = c.astype(float)
    u = np.array(u)
    f = orc.feq(rho, u)
    assert abs(f.sum() - rho) < 1e-14
    assert np.allclose(f @ c, rho * u, atol=1e-15)
    P = np.einsum("i,ia,ib->ab", f, c, c)
    assert np.allclose(P, rho / 3.0 * np.eye(3) + rho * np.outer(u, u), atol=1e-14)


def test_equilibrium_at_rest_is_the_weights(orc):
    _, w, _ = orc.tables()
    assert np.allclose(orc.feq(1.0, [0, 0, 0]), w, atol=0)


@pytest.mark.parametrize("G", [(1e-3, 0, 0), (0.0, -2e-2, 5e-3), (0.3, 0.1, -0.7)])
def test_source_moments(orc, G):
    """Sec. II, Eq. 8: sum_i S_i = 0 and sum_i S_i c_i equals the momentum
    handed to the fluid; the second moment vanishes (no stress input)."""
    c, _, _ = orc.tables()
    c = c.astype(float)
    S = orc.source(G)
    assert abs(S.sum()) < 1e-16
    assert np.allclose(S @ c, np.array(G), atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", S, c, c), 0.0, atol=1e-16)


def _random_state(orc, shape, seed, amp=0.02):
    c, w, _ = orc.tables()
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    return w[:, None, None, None] * (1.0 + amp * rng.standard_normal((19, nz, ny, nx)))


def test_periodic_step_conserves_mass_and_momentum(orc):
    """BGK collision + streaming conserve mass and momentum in a periodic box
    (the collision by construction of feq, streaming by permutation)."""
    c, _, _ = orc.tables()
    shape = (5, 6, 7)
    sim = orc.OracleSim(dict(nx=7, ny=6, nz=5, tau=0.8))
    f0 = _random_state(orc, shape, 1)
    sim.set_populations(f0)
    m0, p0 = f0.sum(), np.einsum("izyx,ia->a", f0, c.astype(float))
    sim.step(25)
    f1 = sim.get_populations()
    assert abs(f1.sum() - m0) < 1e-12 * m0
    assert np.allclose(np.einsum("izyx,ia->a", f1, c.astype(float)), p0, atol=1e-13)


def test_rest_state_is_a_fixed_point_with_walls(orc):
    """f = w (rest, rho = 1) is a fixed point of collision, streaming and
    halfway bounce-back in any geometry; solid sites hold nothing."""
    from paper_0711_2665_gb300 import inputs
    solid = inputs.pore_wall_mask(8, 6, 6, 4, 2)
    sim = orc.OracleSim(dict(nx=8, ny=6, nz=6, tau=1.0), solid)
    sim.step(3)
    f = sim.get_populations()
    _, w, _ = orc.tables()
    assert np.allclose(f[:, solid == 0], w[:, None], atol=1e-15)
    assert np.all(f[:, solid == 1] == 0.0)


def test_streaming_moves_each_population_along_its_link(orc):
    """With omega -> 0 the collision is the identity and one step is pure
    streaming: f_i(x + c_i) = f_i(x) at fluid targets, and a population whose
    target is solid comes back as f_opp(i)(x) (halfway bounce-back)."""
    from paper_0711_2665_gb300 import inputs
    nx, ny, nz = 6, 5, 4
    solid = inputs.pore_wall_mask(nx, ny, nz, 3, 1)
    c, w, opp = orc.tables()
    rng = np.random.default_rng(11)
    f0 = rng.uniform(0.01, 0.1, size=(19, nz, ny, nx)) * (solid == 0)
    sim = orc.OracleSim(dict(nx=nx, ny=ny, nz=nz, tau=1e30), solid)
    sim.set_populations(f0)
    sim.step(1)
    f1 = sim.get_populations()
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        if solid[z, y, x]:
            continue
        for i in range(19):
            tx, ty, tz = (x + c[i, 0]) % nx, (y + c[i, 1]) % ny, (z + c[i, 2]) % nz
            if solid[tz, ty, tx]:
                assert f1[opp[i], z, y, x] == f0[i, z, y, x]
            else:
                assert f1[i, tz, ty, tx] == f0[i, z, y, x]


def test_collision_single_site_relaxation(orc):
    """One site, tau = 1 (omega = 1): the post-collision state is exactly feq
    of the pre-collision moments, so after the (self-)streaming of a 1x1x1
    periodic box the populations equal feq(rho, u)."""
    c, w, _ = orc.tables()
    rng = np.random.default_rng(5)
    f = w * (1 + 0.05 * rng.standard_normal(19))
    sim = orc.OracleSim(dict(nx=1, ny=1, nz=1, tau=1.0))
    sim.set_populations(f)
    sim.step(1)
    rho = f.sum()
    u = (f @ c.astype(float)) / rho
    assert np.allclose(sim.get_populations().reshape(-1), orc.feq(rho, u), atol=1e-15)


def test_relaxation_rate_of_a_nonconserved_moment(orc):
    """In a 1x1x1 box a non-conserved moment m = sum f_i c_ix c_iy relaxes as
    m - m_eq -> (1 - omega)(m - m_eq) per step."""
    c, w, _ = orc.tables()
    c = c.astype(float)
    rng = np.random.default_rng(7)
    f = w * (1 + 0.05 * rng.standard_normal(19))
    tau = 0.7
    sim = orc.OracleSim(dict(nx=1, ny=1, nz=1, tau=tau))
    sim.set_populations(f)
    rho = f.sum()
    u = (f @ c) / rho
    pxy = lambda g: float(np.sum(g * c[:, 0] * c[:, 1]))
    meq = rho * u[0] * u[1]
    d0 = pxy(f) - meq
    sim.step(1)
    d1 = pxy(sim.get_populations().reshape(-1)) - meq
    assert abs(d1 - (1 - 1 / tau) * d0) < 1e-15
