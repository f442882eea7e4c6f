"""Pins of the oracle's fluctuating lattice Boltzmann (the stochastic term F_i of
Sec. II, Eq. 4, in the moment-space form of the cited work of Adhikari et al.).

* The 19 modes are an orthogonal basis under the lattice weights, in exact
  rational arithmetic; modes 0..3 are density and momentum.
* The fluctuation touches no conserved mode: mass and momentum of a periodic
  box stay constant to rounding, and mass with a wall too.
* Equipartition: in equilibrium every site's populations fluctuate with
  covariance mu w_i delta_ij (mu = rho kT / c_s^2), so <(rho u_a)^2> = rho kT,
  <drho^2> = 3 rho kT and a shear mode has mu b_k, at any tau.
* The site noise has zero mean and unit variance and is independent of the
  bead noise (different counters of the same generator).
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_0711_2665_gb300 import inputs

KT = 1e-4


def test_mode_basis_is_orthogonal(orc):
    c, _, _ = orc.tables()
    w = [Fraction(1, 3)] + [Fraction(1, 18)] * 6 + [Fraction(1, 36)] * 12
    E = [[Fraction(orc.mode(k, c[i])).limit_denominator(1) for i in range(19)] for k in range(19)]
    for k in range(19):
        for l in range(19):
            g = sum(w[i] * E[k][i] * E[l][i] for i in range(19))
            if k == l:
                assert g > 0
            else:
                assert g == 0, (k, l, g)
    assert all(E[0][i] == 1 for i in range(19))
    for a in range(3):
        assert all(E[1 + a][i] == c[i][a] for i in range(19))


@pytest.mark.parametrize("wall", [False, True])
def test_fluctuation_conserves_mass_and_momentum(orc, wall):
    dims = (12, 10, 10)
    solid = inputs.pore_wall_mask(*dims, 6, 3) if wall else None
    s = orc.OracleSim(dict(nx=dims[0], ny=dims[1], nz=dims[2], tau=0.8, n_beads=0, lb_kT=KT, seed=3), solid)
    o0 = s.observables()
    s.step(20)
    o1 = s.observables()
    assert abs(o1["mass"] - o0["mass"]) < 1e-12 * o0["mass"]
    if not wall:
        for a in ("x", "y", "z"):
            assert abs(o1["p_fluid_" + a] - o0["p_fluid_" + a]) < 1e-13
    f = s.get_populations()
    assert np.abs(f.sum(0) - 1.0)[(solid == 0) if wall else slice(None)].max() > 1e-4  # it does fluctuate


@pytest.mark.parametrize("tau", [0.6, 1.0])
def test_equipartition(orc, tau):
    s = orc.OracleSim(dict(nx=16, ny=16, nz=16, tau=tau, n_beads=0, lb_kT=KT, seed=5))
    s.step(150)
    c, w, _ = orc.tables()
    b7 = np.sum(w * (c[:, 0] * c[:, 1]) ** 2)
    acc = np.zeros(5)
    n = 60
    for _ in range(n):
        s.step(1)
        f = s.get_populations()
        rho = f.sum(0)
        j = np.tensordot(c.T.astype(float), f, 1)
        m7 = np.tensordot(c[:, 0] * c[:, 1], f, 1)
        acc += [np.mean(j[0] ** 2), np.mean(j[1] ** 2), np.mean(j[2] ** 2), np.mean((rho - 1) ** 2), np.mean(m7 ** 2)]
    acc /= n
    assert np.allclose(acc[:3] / KT, 1.0, atol=0.03), acc[:3] / KT
    assert acc[3] / (3 * KT) == pytest.approx(1.0, abs=0.03)
    assert acc[4] / (3 * KT * b7) == pytest.approx(1.0, abs=0.03)


def test_site_noise_statistics(orc):
    z = np.array([orc.fluid_noise(9, 2, site, 17) for site in range(20000)])
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / z.size)
    zb = np.array([orc.gauss3(9, 2, site, 17, 0) for site in range(20000)])
    r = np.corrcoef(z[:, 0], zb[:, 0])[0, 1]
    assert abs(r) < 5 / np.sqrt(20000)
