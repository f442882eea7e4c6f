"""Failure detection of the step, with every fault made on the host.

The particle kernel keeps fixed-capacity lists in shared memory: at most 32
bead neighbours (within the list radius 2^(1/6) sigma + skin) and 12 solid
sites (within 2^(1/6) sigma_w + skin/2) per bead.  A state that needs more
is clamped and latched as a capacity error, which lbmd_check reports as
LBMD_ERR_CAPACITY; a non-finite bead or fluid state is latched as
LBMD_ERR_NONFINITE.  The states below are built on the host: crowded beads
with the pair forces switched off (eps = 0) so that nothing else goes wrong,
and a NaN planted in one bead's velocity or position.  Positions that are
not finite are mapped to site 0 before any lattice index is formed, so the
NaN cases index only inside the lattice.  The bounded device waits are
tested through lbmd_set_wait_probe: a wait on an mbarrier phase that nothing
completes, with no copy in flight, runs out after 1 ms (LBMD_ERR_TIMEOUT).
"""
import numpy as np
import pytest

from gpu_helpers import small_workload
from paper_0711_2665_gb300 import lbmd

pytestmark = pytest.mark.gpu

CAPACITY, NONFINITE, TIMEOUT = 5, 3, 4


def _quiet(**kw):
    """16^3 periodic box, no forces at all on the beads (no bonds, bending,
    WCA, field, friction or noise), so that crowding cannot blow up."""
    base = dict(nx=16, ny=16, nz=16, wall_x=-1, pore_h=0, k_bond=0.0, kappa_bend=0.0, lj_eps=0.0,
                wall_eps=0.0, E=0.0, gamma=0.0, kT=0.0)
    base.update(kw)
    return small_workload(**base)


def _status_after(sim, steps=1):
    sim.step(steps)
    with pytest.raises(lbmd.LbmdError) as e:
        sim.check()
    obs = sim.observables()[0]
    return e.value.status, obs["status"]


def test_neighbour_list_overflow_is_reported():
    """40 beads on a 4 x 4 x 3 grid of spacing 0.35: every pair lies within
    1.64 < 1.72 of each other, so each bead has at least 37 non-bonded
    neighbours, more than the 32 a list holds."""
    g = np.stack(np.meshgrid(np.arange(4), np.arange(4), np.arange(3), indexing="ij"), -1).reshape(-1, 3)[:40]
    r = 8.0 + 0.35 * g.astype(np.float64)
    d = np.linalg.norm(r[:, None] - r[None], axis=-1)
    assert d.max() < 2 ** (1 / 6) + 0.6 and d[d > 0].min() > 0.3
    w = _quiet(n_beads=40)
    sim = lbmd.Simulation(w, np.zeros((16, 16, 16), np.uint8), [0, 40], r)
    st, obs_st = _status_after(sim)
    assert st == CAPACITY and obs_st == CAPACITY
    r1, v1 = sim.get_beads()
    assert np.all(np.isfinite(r1)) and np.all(np.isfinite(v1))


def test_wall_list_overflow_is_reported():
    """One bead 0.004 from the centre site of a solid 3 x 3 x 3 block: 19
    solid sites (the centre, its 6 faces and 12 edges, at squared distances
    below 2.01) lie within the wall-list radius 2^(1/6) + 0.3 = 1.42 (squared
    2.02), more than the 12 a list holds.  (Off the centre so that no
    distance is zero: with eps = 0 the WCA term is 0 times a finite number.)"""
    solid = np.zeros((16, 16, 16), np.uint8)
    solid[6:9, 6:9, 6:9] = 1
    r = np.array([[7.001, 7.002, 7.003]])
    d2 = ((np.argwhere(solid)[:, ::-1] - r) ** 2).sum(1)
    assert (d2 < (2 ** (1 / 6) + 0.3) ** 2).sum() == 19 and d2.min() > 1e-6
    w = _quiet(n_beads=1)
    sim = lbmd.Simulation(w, solid, [0, 1], r)
    st, obs_st = _status_after(sim)
    assert st == CAPACITY and obs_st == CAPACITY


def test_crowding_within_capacity_is_not_reported():
    """The same box with 12 beads spaced 0.35 (11 neighbours each) and one
    bead beside (not inside) the solid block: no error."""
    solid = np.zeros((16, 16, 16), np.uint8)
    solid[6:9, 6:9, 6:9] = 1
    g = np.stack(np.meshgrid(np.arange(3), np.arange(2), np.arange(2), indexing="ij"), -1).reshape(-1, 3)
    r = np.vstack([2.0 + 0.35 * g.astype(np.float64), [[10.0, 7.0, 7.0]]])
    w = _quiet(n_beads=13)
    sim = lbmd.Simulation(w, solid, [0, 13], r)
    sim.step(2)
    sim.check()
    assert sim.observables()[0]["status"] == 0


@pytest.mark.parametrize("what", ["v", "r"])
def test_nonfinite_bead_state_is_reported(what):
    """A NaN planted in one bead's velocity or position of a normal coupled
    case is latched by the particle kernel and reported."""
    w = small_workload()
    from paper_0711_2665_gb300 import workloads
    inp = workloads.build_inputs(w)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    sim.step(2)
    r, v = sim.get_beads()
    if what == "v":
        v[5, 1] = np.nan
    else:
        r[5, 0] = np.nan
    sim.set_beads(r, v)
    st, obs_st = _status_after(sim)
    assert st == NONFINITE and obs_st == NONFINITE


def test_bounded_wait_that_runs_out_is_reported():
    """The tensor-copy lattice pass told to wait on an mbarrier phase that
    nothing completes (before it issues any copy) gives up after 1 ms,
    latches the timeout and returns: lbmd_check reports LBMD_ERR_TIMEOUT and
    the context stays usable, a fresh handle stepping exactly like one that
    never waited.  Two ordinary steps first leave both population buffers
    finite, so the skipped pass leaves a finite (if invalid) state."""
    from paper_0711_2665_gb300 import workloads
    w = small_workload()
    inp = workloads.build_inputs(w)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    sim.set_tiles(0, 4)
    sim.step(2)
    sim.check()
    sim.set_wait_probe(True)
    st, obs_st = _status_after(sim)
    assert st == TIMEOUT and obs_st == TIMEOUT
    sim.close()
    runs = []
    for tiles in ((0, 4), (4, 4)):
        s2 = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
        s2.set_tiles(*tiles)
        s2.step(3)
        s2.check()
        runs.append(s2.get_deviations())
        s2.close()
    assert np.array_equal(runs[0], runs[1])
