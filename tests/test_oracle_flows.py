"""Hydrodynamic pins of the oracle: shear-wave decay, Poiseuille flow, and the
conservation laws of the coupled step.

* Shear wave: the decay factor per step of u_y = A sin(2 pi x / L) must equal
  the eigenvalue of the linearised LBGK operator at k = 2 pi / L, computed here
  independently as a 19x19 Fourier-space matrix, and approach the
  Navier-Stokes rate nu k^2 with nu = c_s^2 (tau - 1/2) (the viscosity law of
  Sec. II read with c_s^2 = 1/3).
* Poiseuille flow between halfway bounce-back walls driven by a uniform body
  force: the steady profile's second difference equals -g / nu.
* Conservation: mass in any geometry; fluid + bead momentum in a periodic box
  without walls; with the pore field, momentum grows by exactly N E per step
  while the beads sit in the channel.
"""
import numpy as np
import pytest

from paper_0711_2665_gb300 import inputs


def _linear_lbgk_eigs(c, w, tau, k):
    """Eigen-decomposition of one linearised LBGK step about rest for a
    perturbation exp(i k x): streaming e^{-i k c_x} after collision
    (1 - omega) I + omega Pi, with Pi_ij = w_i (1 + 3 c_i . c_j)."""
    omega = 1.0 / tau
    c = c.astype(float)
    Pi = w[:, None] * (1.0 + 3.0 * c @ c.T)
    C = (1.0 - omega) * np.eye(19) + omega * Pi
    D = np.diag(np.exp(-1j * k * c[:, 0]))
    return np.linalg.eig(D @ C)


@pytest.mark.parametrize("tau,nx", [(0.8, 32), (1.0, 24), (0.6, 40)])
def test_shear_wave_decay_matches_linear_eigenvalue(orc, tau, nx):
    c, w, _ = orc.tables()
    k = 2 * np.pi / nx
    A = 1e-6
    sim = orc.OracleSim(dict(nx=nx, ny=1, nz=1, tau=tau))
    u0 = inputs.shear_wave_velocity(nx, 1, 1, A)
    sim.init_fluid(None, u0)
    x = np.arange(nx)
    s = np.sin(k * x)

    def amp():
        _, u = sim.moments()
        return 2.0 / nx * float(u[1, 0, 0, :] @ s)

    sim.step(60)  # non-hydrodynamic modes die as |1 - omega|^t
    a1 = amp()
    n = 400
    sim.step(n)
    a2 = amp()
    rate = (a2 / a1) ** (1.0 / n)
    # the shear mode: eigenvector dominated by the y-momentum moment
    lam, vec = _linear_lbgk_eigs(c, w, tau, k)
    jy = np.abs(c[:, 1].astype(float) @ vec)
    lam_shear = lam[np.argmax(jy)]
    assert abs(lam_shear.imag) < 1e-12
    assert abs(rate - lam_shear.real) < 1e-5 * abs(1 - lam_shear.real)
    # Navier-Stokes limit: 1 - rate ~ nu k^2 to O(k^2) relative
    nu = (tau - 0.5) / 3.0
    assert abs(-np.log(rate) - nu * k * k) < 0.03 * nu * k * k


def _poiseuille(orc, tau, ny, g, steps):
    solid = inputs.slab_walls_mask(1, ny, 1, axis="y")
    sim = orc.OracleSim(dict(nx=1, ny=ny, nz=1, tau=tau, body_force=(g, 0.0, 0.0)), solid)
    sim.step(steps)
    _, u = sim.moments()
    return u[0, 0, :, 0]


@pytest.mark.parametrize("tau", [0.8, 1.0])
def test_poiseuille_curvature(orc, tau):
    """Steady plane Poiseuille flow: u(y+1) - 2u(y) + u(y-1) = -g / nu in the
    bulk, with nu = (tau - 1/2)/3, and the profile is symmetric."""
    ny, g = 17, 1e-6
    nu = (tau - 0.5) / 3.0
    u = _poiseuille(orc, tau, ny, g, 12000)
    fl = u[1:]  # fluid rows 1..ny-1
    d2 = fl[2:] - 2 * fl[1:-1] + fl[:-2]
    assert np.allclose(d2, -g / nu, rtol=1e-8, atol=0)
    assert np.allclose(fl, fl[::-1], rtol=1e-10)


def test_poiseuille_wall_location_at_the_magic_tau(orc):
    """For BGK with halfway bounce-back the no-slip wall sits exactly halfway
    between the solid plane and the first fluid row when (tau - 1/2)^2 = 3/16;
    then the parabola fitted to the profile vanishes at y = 1/2 and y = ny - 1/2.
    The source of Sec. II, Eq. 9 adds the force after the moments are taken, so
    the fluid's mean velocity over the step is u + g/(2 rho): that is the
    profile whose zeros locate the wall (rho = 1 here)."""
    tau = 0.5 + np.sqrt(3.0) / 4.0
    ny, g = 17, 1e-6
    u = _poiseuille(orc, tau, ny, g, 12000) + 0.5 * g
    y = np.arange(1, ny, dtype=float)
    coef = np.polyfit(y, u[1:], 2)
    roots = np.sort(np.roots(coef).real)
    assert abs(roots[0] - 0.5) < 1e-6 and abs(roots[1] - (ny - 0.5)) < 1e-6


def _coupled_sim(orc, solid=None, **kw):
    p = dict(nx=12, ny=10, nz=10, tau=0.8, n_beads=6, k_bond=100.0, r0=1.0, kappa_bend=1e-3,
             lj_sigma=1.0, lj_eps=1.0, wall_sigma=1.0, wall_eps=1.0, E=0.0, gamma=0.1,
             kT=1e-4, md_outer=5, md_inner=20, seed=123, wall_x=-1, pore_h=3)
    p.update(kw)
    sim = orc.OracleSim(p, solid)
    return sim, p


def _total_momentum(o):
    return np.array([o["p_fluid_x"] + o["p_beads_x"], o["p_fluid_y"] + o["p_beads_y"],
                     o["p_fluid_z"] + o["p_beads_z"]])


@pytest.mark.parametrize("kT", [0.0, 1e-4])
def test_momentum_conserved_fluid_plus_beads(orc, kT):
    """No walls and no field: friction and noise only move momentum between
    beads and fluid, bonds/bending/WCA are internal, so the total is constant."""
    sim, p = _coupled_sim(orc, kT=kT)
    rng = np.random.default_rng(3)
    r = inputs.chain_walk(6, (12, 10, 10), -1, np.zeros((10, 10, 12), np.uint8), 9)
    v = 0.05 * rng.standard_normal((6, 3))
    sim.set_beads(r, v)
    P0 = _total_momentum(sim.observables())
    sim.step(30)
    P1 = _total_momentum(sim.observables())
    assert np.all(np.abs(P0) > 1e-3)
    assert np.allclose(P1, P0, atol=1e-13)
    # and momentum did move between the two
    o = sim.observables()
    assert abs(o["p_fluid_x"]) > 1e-3


def test_mass_conserved_with_wall_and_beads(orc):
    solid = inputs.pore_wall_mask(12, 10, 10, 6, 3)
    sim, p = _coupled_sim(orc, solid=solid, wall_x=6, E=0.05)
    r = inputs.chain_walk(6, (12, 10, 10), 6, solid, 4)
    sim.set_beads(r)
    m0 = sim.observables()["mass"]
    sim.step(30)
    m1 = sim.observables()["mass"]
    assert m0 == pytest.approx(int((solid == 0).sum()), rel=1e-15)
    assert abs(m1 - m0) < 1e-12 * m0


def test_field_impulse_is_exactly_N_E_per_step(orc):
    """Beads held inside the pore channel (no solid wall, wall_x only marks
    the channel) receive q E per unit time each; the total momentum of fluid
    + beads therefore grows by N E per LB step."""
    E = 1e-3
    sim, p = _coupled_sim(orc, n_beads=2, wall_x=6, E=E, kT=0.0, kappa_bend=0.0)
    r = np.array([[5.6, 5.0, 5.0], [6.4, 5.2, 5.0]])  # pore centre is (6, 5, 5)
    sim.set_beads(r)
    P0 = _total_momentum(sim.observables())
    n = 3
    sim.step(n)
    rr, _ = sim.get_beads()
    assert np.all(np.abs(rr[:, 0] - 6) <= 1.5)
    P1 = _total_momentum(sim.observables())
    assert np.allclose(P1 - P0, [2 * E * n, 0, 0], atol=1e-14)
