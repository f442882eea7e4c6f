"""Pins of the oracle's observables (Sec. III global sums; Sec. IV.A-C) by
closed forms of hand-placed configurations:

* the radius of gyration of n beads evenly spaced a unit apart on a line is
  sqrt((n^2 - 1) / 12) (the variance of 0 .. n-1), and it does not move
  under a translation;
* a bead counts as translocated exactly when its unwrapped x exceeds
  wall_x + 1/2, and each part's radius is that of its own beads;
* the field's work rate is E v_x for a bead inside the pore channel
  (|x - wall_x| <= 3/2, y and z within the pore padded by half a site) and 0
  outside it;
* in a uniform flow u0 the fluid velocity at every bead is u0, so the
  friction work rate is gamma u0 . sum v;
* the bead momentum is the sum of the velocities and the centre of mass the
  mean position."""
import numpy as np
import pytest

NX, NY, NZ, WALL = 24, 12, 12, 12
C = 6.0  # centre of the 3x3 pore: fluid rows 5, 6, 7 of the wall plane


def _sim(orc, n, solid=None, **kw):
    p = dict(nx=NX, ny=NY, nz=NZ, tau=0.8, n_beads=n, k_bond=100.0, r0=1.0, kappa_bend=1e-3,
             lj_sigma=1.0, lj_eps=1.0, wall_sigma=1.0, wall_eps=1.0, E=0.05, gamma=0.1, kT=0.0,
             md_outer=5, md_inner=20, seed=1, wall_x=WALL, pore_h=3)
    p.update(kw)
    return orc.OracleSim(p, solid)


def _line(n, x, y0=2.0, z=3.0):
    return np.array([[x, y0 + k, z] for k in range(n)], dtype=float)


@pytest.mark.parametrize("n", [1, 2, 7, 10])
def test_straight_chain(orc, n):
    sim = _sim(orc, n)
    r = _line(n, 4.0)
    v = np.array([[0.01 * k, -0.02, 0.003 * k * k] for k in range(n)])
    sim.set_beads(r, v)
    o = sim.observables()
    assert o["rg_untranslocated"] == pytest.approx(np.sqrt((n * n - 1) / 12.0), rel=1e-14, abs=1e-14)
    assert o["rg_translocated"] == 0.0 and o["n_translocated"] == 0.0
    assert (o["com_x"], o["com_y"], o["com_z"]) == pytest.approx((4.0, 2.0 + (n - 1) / 2.0, 3.0), rel=1e-14)
    assert (o["p_beads_x"], o["p_beads_y"], o["p_beads_z"]) == pytest.approx(tuple(v.sum(axis=0)), rel=1e-14)
    # a translation (also across periodic images: unwrapped x) leaves the radius
    sim.set_beads(r + np.array([-30.0, 5.5, -1.25]), v)
    assert sim.observables()["rg_untranslocated"] == pytest.approx(np.sqrt((n * n - 1) / 12.0), rel=1e-12)


def test_split_chain_and_threshold(orc):
    k, m = 4, 6  # translocated, untranslocated
    r = np.concatenate([_line(k, WALL + 3.0), _line(m, WALL - 3.0)])
    sim = _sim(orc, k + m)
    sim.set_beads(r)
    o = sim.observables()
    assert o["n_translocated"] == k
    assert o["rg_translocated"] == pytest.approx(np.sqrt((k * k - 1) / 12.0), rel=1e-14)
    assert o["rg_untranslocated"] == pytest.approx(np.sqrt((m * m - 1) / 12.0), rel=1e-14)
    # the threshold itself is not past the wall; just beyond it is
    for x, past in ((WALL + 0.5, 0), (WALL + 0.5 + 1e-9, 1), (WALL + 0.5 - 1e-9, 0), (WALL + 0.5 + 24.0, 1)):
        one = _sim(orc, 1)
        one.set_beads(np.array([[x, 2.0, 3.0]]))
        assert one.observables()["n_translocated"] == past, x


def test_field_work_rate(orc):
    E = 0.05
    vx = 0.3
    inside = [(WALL, C, C), (WALL + 1.5, C, C), (WALL - 1.5, C + 1.5, C - 1.5), (WALL + 1.4 + NX, C, C)]
    outside = [(WALL + 1.6, C, C), (WALL, C + 1.6, C), (WALL, C, C - 1.6), (WALL - 3.0, C, C)]
    for pos, expect in [(p, E * vx) for p in inside] + [(p, 0.0) for p in outside]:
        sim = _sim(orc, 1, E=E)
        sim.set_beads(np.array([pos], dtype=float), np.array([[vx, 0.2, -0.1]]))
        assert sim.observables()["dWE_dt"] == pytest.approx(expect, rel=1e-14, abs=1e-300), pos


def test_friction_work_rate_in_uniform_flow(orc):
    n, gamma = 5, 0.1
    u0 = np.array([0.012, -0.004, 0.007])
    sim = _sim(orc, n, wall_x=-1, gamma=gamma)
    ns = NX * NY * NZ
    sim.init_fluid(None, np.repeat(u0[:, None], ns, axis=1))
    rng = np.random.default_rng(5)
    r = _line(n, 7.3, 1.6, 4.4)
    v = 0.05 * rng.standard_normal((n, 3))
    sim.set_beads(r, v)
    o = sim.observables()
    assert o["dWH_dt"] == pytest.approx(gamma * float(u0 @ v.sum(axis=0)), rel=1e-12)
    # no flow, no friction work
    still = _sim(orc, n, wall_x=-1, gamma=gamma)
    still.set_beads(r, v)
    assert still.observables()["dWH_dt"] == pytest.approx(0.0, abs=1e-15)
