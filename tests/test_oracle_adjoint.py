"""Pins of the oracle's discrete adjoint (reverse mode of the coupled step).

The adjoint is checked against the oracle's own forward step, never against
itself:

* the gradient of L = mean x(K) - mean x(0) with respect to gamma, E and every
  initial bead coordinate equals the FP64 central finite difference of the
  forward run (h = 1e-4), on a small lattice with a wall, a pore, noise and a
  chain partly inside the pore channel; entries whose +h and -h runs differ in
  a non-differentiable event (a kick inside / outside the channel, a bead in
  another lattice cell) are left out and counted;
* one step's adjoint passes the dot-product test <lam, J d> = <J^T lam, d>
  with J d from a central difference of the forward step along a random
  direction d of (f, r, v);
* a single bead under a constant field with no friction or noise moves as
  x = x0 + v0 t + E t^2 / 2 exactly (velocity Verlet is exact for constant
  force): dL/dE = K^2 / 2, dL/dv0_x = K, dL/dr0 = 0;
* with gamma = 0 the beads never feel the fluid: dL/df0 = 0 exactly;
* with only internal forces the centre of mass drifts freely:
  L = K mean(v0_x), so dL/dr0 = 0 and dL/dv0_x = K / N.
"""
import numpy as np
import pytest

from paper_0711_2665_gb300 import inputs

DIMS = (20, 12, 12)
WALL = 10


def _params(**kw):
    p = dict(nx=DIMS[0], ny=DIMS[1], nz=DIMS[2], tau=0.8, wall_x=WALL, pore_h=3, n_beads=6,
             kappa_bend=1e-3, E=0.1, gamma=0.1, kT=1e-4, seed=7)
    p.update(kw)
    return p


def _chain(n=6, seed=3, shift=0.3):
    solid = inputs.pore_wall_mask(*DIMS, WALL, 3)
    r0 = inputs.chain_walk(n, DIMS, WALL, solid, seed)
    r0[:, 0] += shift  # the first beads sit inside the pore channel
    r0[:, 1:] += 0.137  # off the cell faces, where the trilinear weights have a kink
    return solid, r0


def _loss(orc, params, solid, r0, K, v0=None):
    s = orc.OracleSim(params, solid)
    s.set_beads(r0, v0)
    x0 = r0[:, 0].mean()
    s.step(K)
    return s.get_beads()[0][:, 0].mean() - x0, s.event_counts()


def test_gradient_matches_central_differences(orc):
    K, h = 6, 1e-4
    P = _params()
    solid, r0 = _chain()
    g = orc.adjoint(P, solid, r0, K)
    loss, _ = _loss(orc, P, solid, r0, K)
    assert g["loss"] == pytest.approx(loss, rel=1e-14, abs=1e-15)
    skipped = 0
    for name in ("gamma", "E"):
        Pp, Pm = dict(P), dict(P)
        Pp[name] += h
        Pm[name] -= h
        (lp, ep), (lm, em) = _loss(orc, Pp, solid, r0, K), _loss(orc, Pm, solid, r0, K)
        fd = (lp - lm) / (2 * h)
        if ep[1] != em[1]:
            skipped += 1
            continue
        # the field derivative tolerates a flipped channel kick: it moves L by
        # O(E dt^2) while E itself moves it by O(K^2) per unit E
        assert g["d" + name] == pytest.approx(fd, rel=2e-5), name
    scale = np.abs(g["dr0"]).max()
    for i in range(r0.shape[0]):
        for a in range(3):
            rp, rm = r0.copy(), r0.copy()
            rp[i, a] += h
            rm[i, a] -= h
            (lp, ep), (lm, em) = _loss(orc, P, solid, rp, K), _loss(orc, P, solid, rm, K)
            if ep != em:
                skipped += 1
                continue
            fd = (lp - lm) / (2 * h)
            assert abs(g["dr0"][i, a] - fd) <= 1e-3 * scale + 1e-3 * abs(fd), (i, a, g["dr0"][i, a], fd)
    assert skipped <= 2


def test_step_adjoint_dot_product(orc):
    P = _params(kappa_bend=0.7)
    solid, r0 = _chain()
    rng = np.random.default_rng(11)
    s0 = orc.OracleSim(P, solid)
    s0.set_beads(r0)
    s0.step(2)  # a state with a moving fluid and moving beads
    f = s0.get_populations().copy()
    r, v = s0.get_beads()
    fluid = (solid.reshape(DIMS[::-1]) == 0)
    df = rng.normal(size=f.shape) * fluid[None] * 1e-3
    dr = rng.normal(size=r.shape) * 1e-2
    dv = rng.normal(size=v.shape) * 1e-2
    lf = rng.normal(size=f.shape) * fluid[None]
    lr = rng.normal(size=r.shape)
    lv = rng.normal(size=v.shape)

    def forward(eps):
        s = orc.OracleSim(P, solid)
        s.set_populations(f + eps * df)
        s.set_beads(r + eps * dr, v + eps * dv)
        s.set_step(2)
        s.step(1)
        rr, vv = s.get_beads()
        return s.get_populations(), rr, vv

    eps = 1e-5
    fp, rp, vp = forward(eps)
    fm, rm, vm = forward(-eps)
    lhs = (np.sum(lf * (fp - fm)) + np.sum(lr * (rp - rm)) + np.sum(lv * (vp - vm))) / (2 * eps)
    s = orc.OracleSim(P, solid)
    s.set_populations(f)
    s.set_beads(r, v)
    s.set_step(2)
    af, ar, av, _ = s.step_adjoint(lf, lr, lv)
    rhs = np.sum(af * df) + np.sum(ar * dr) + np.sum(av * dv)
    assert rhs == pytest.approx(lhs, rel=1e-6)
    # the state is advanced like a forward step
    fa = s.get_populations()
    f1, _, _ = forward(0.0)
    assert np.array_equal(fa, f1)


def test_constant_field_closed_form(orc):
    K, E = 10, 0.01
    c = DIMS[1] // 2
    P = _params(n_beads=1, gamma=0.0, kT=0.0, E=E)
    solid = inputs.pore_wall_mask(*DIMS, WALL, 3)
    r0 = np.array([[WALL - 1.0, c, c]])
    g = orc.adjoint(P, solid, r0, K)
    assert g["loss"] == pytest.approx(E * K * K / 2, rel=1e-12)
    assert g["dE"] == pytest.approx(K * K / 2, rel=1e-12)
    assert g["dv0"][0, 0] == pytest.approx(K, rel=1e-12)
    assert np.abs(g["dr0"]).max() < 1e-12


def test_no_friction_no_fluid_gradient(orc):
    P = _params(gamma=0.0, kT=0.0)
    solid, r0 = _chain()
    g = orc.adjoint(P, solid, r0, 4, want_df0=True)
    assert np.all(g["df0"] == 0.0)


def test_internal_forces_only_translation(orc):
    K, N = 5, 6
    P = _params(gamma=0.0, kT=0.0, E=0.0, wall_x=-1, kappa_bend=0.7)
    _, r0 = _chain()
    rng = np.random.default_rng(5)
    v0 = 0.01 * rng.normal(size=r0.shape)
    g = orc.adjoint(P, None, r0, K, v0=v0)
    assert g["loss"] == pytest.approx(K * v0[:, 0].mean(), rel=1e-10)
    assert np.abs(g["dr0"]).max() < 1e-8
    assert np.allclose(g["dv0"][:, 0], K / N, rtol=1e-8)
    assert np.abs(g["dv0"][:, 1:]).max() < 1e-8


def test_channel_trace_replay_and_frozen_differences(orc):
    """Replaying a recorded pore-channel trace reproduces the run bit for bit;
    with the trace held, central differences over a horizon where plain
    differences cross field events agree with the adjoint."""
    K, h = 12, 1e-4
    P = _params()
    solid, r0 = _chain()
    N, M = r0.shape[0], P.get("md_outer", 5)
    trace = np.zeros(K * 2 * M * N, dtype=np.int32)
    s = orc.OracleSim(P, solid)
    s.set_beads(r0)
    s.channel_trace(1, trace)
    s.step(K)
    rec_r, rec_v = s.get_beads()
    assert trace.sum() == s.event_counts()[0] > 0
    s2 = orc.OracleSim(P, solid)
    s2.set_beads(r0)
    s2.channel_trace(2, trace)
    s2.step(K)
    r2, v2 = s2.get_beads()
    assert np.array_equal(r2, rec_r) and np.array_equal(v2, rec_v)
    assert np.array_equal(s2.get_populations(), s.get_populations())

    def frozen(params, r):
        q = orc.OracleSim(params, solid)
        q.set_beads(r)
        q.channel_trace(2, trace)
        x0 = r[:, 0].mean()
        q.step(K)
        return q.get_beads()[0][:, 0].mean() - x0

    g = orc.adjoint(P, solid, r0, K)
    for name in ("gamma", "E"):
        Pp, Pm = dict(P), dict(P)
        Pp[name] += h
        Pm[name] -= h
        fd = (frozen(Pp, r0) - frozen(Pm, r0)) / (2 * h)
        assert g["d" + name] == pytest.approx(fd, rel=1e-4), name
    scale = np.abs(g["dr0"]).max()
    for i, a in ((0, 0), (1, 2), (4, 1)):
        rp, rm = r0.copy(), r0.copy()
        rp[i, a] += h
        rm[i, a] -= h
        fd = (frozen(P, rp) - frozen(P, rm)) / (2 * h)
        assert abs(g["dr0"][i, a] - fd) <= 1e-3 * scale + 1e-3 * abs(fd)
