"""The two variants of the step on the GPU against the FP64 oracle:
nearest-grid-point coupling (interp = 1, the paper's scheme) and the stochastic
position Verlet cycle (integrator = 1, Sec. II, Eq. SPValgo nested).  One step
from a developed state within the parity tolerances (see test_gpu_parity.py);
fluid + bead momentum conserved; the NGP adjoint against the oracle adjoint;
the adjoint refuses the SPV cycle."""
import numpy as np
import pytest

import oracle
from gpu_helpers import load_state, make_pair, rel_err, small_workload, to_f32_state
from paper_0711_2665_gb300 import lbmd, workloads

pytestmark = pytest.mark.gpu

VARIANTS = [dict(interp=1), dict(integrator=1), dict(interp=1, integrator=1)]


@pytest.mark.parametrize("variant", VARIANTS)
def test_one_step_from_developed_state(variant):
    w = small_workload(**variant)
    sim, orc, inp = make_pair(w)
    orc.step(6)
    f32, r, v = to_f32_state(orc)
    load_state(sim, orc, f32, r, v, 6)
    r_before = r.copy()
    sim.step(1)
    orc.step(1)
    assert rel_err(sim.get_populations()[0], orc.get_populations()) <= 1e-5
    r_g, v_g = sim.get_beads()
    r_o, v_o = orc.get_beads()
    floor = w["k_bond"] * 2.0 ** -24
    assert np.abs(r_g - r_o).max() <= 1e-5 * np.abs(r_o - r_before).max() + 1e-6 + floor
    assert np.abs(v_g - v_o).max() <= 1e-5 * np.abs(v_o).max() + floor
    up_g, J_g = sim.get_coupling()
    up_o, J_o = orc.last_coupling()
    assert rel_err(J_g, J_o) <= 1e-4, rel_err(J_g, J_o)


@pytest.mark.parametrize("variant", VARIANTS)
def test_momentum_conserved(variant):
    w = small_workload(wall_x=-1, E=0.0, kT=1e-4, n_beads=16, **variant)
    inp = workloads.build_inputs(w)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    rng = np.random.default_rng(4)
    sim.set_beads(inp["r0"], 0.05 * rng.standard_normal(inp["r0"].shape))

    def total(o):
        return np.array([o["p_fluid_x"] + o["p_beads_x"], o["p_fluid_y"] + o["p_beads_y"],
                         o["p_fluid_z"] + o["p_beads_z"]])

    P0 = total(sim.observables()[0])
    sim.step(20)
    P1 = total(sim.observables()[0])
    assert np.abs(P1 - P0).max() < 1e-4 * np.abs(P0).max()


def test_nearest_grid_point_adjoint_matches_oracle():
    K = 6
    w = small_workload(nx=40, ny=20, nz=12, wall_x=20, n_beads=10, kappa_bend=1e-3, interp=1)
    inp = workloads.build_inputs(w)
    r0 = inp["r0"].copy()
    r0[0] += (0.4, 0.137, 0.137)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], r0)
    g = sim.adjoint(K, 4)
    o = oracle.adjoint(workloads.oracle_params(w, 0, r0.shape[0]), inp["solid"], r0, K)
    assert g["dgamma"][0] == pytest.approx(o["dgamma"], rel=1e-3)
    assert g["dE"][0] == pytest.approx(o["dE"], rel=1e-3)
    scale = np.abs(o["dr0"]).max()
    assert np.all(np.abs(g["dr0"] - o["dr0"]) <= 1e-3 * scale + 1e-3 * np.abs(o["dr0"]))


def test_adjoint_refuses_spv():
    w = small_workload(integrator=1)
    inp = workloads.build_inputs(w)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    with pytest.raises(lbmd.LbmdError) as e:
        sim.adjoint_bytes(4, 2)
    assert e.value.status == 1


# ---------------------------------------------------------------------------
# fluctuating lattice Boltzmann (lb_kT > 0)
# ---------------------------------------------------------------------------
LB_KT = 1e-4


def test_fluctuating_one_step_matches_oracle():
    """Same Philox normals per site and step on both sides: one coupled step
    from a developed state within the parity tolerance."""
    w = small_workload(lb_kT=LB_KT)
    sim, orc, inp = make_pair(w)
    orc.step(5)
    f32, r, v = to_f32_state(orc)
    load_state(sim, orc, f32, r, v, 5)
    sim.step(1)
    orc.step(1)
    assert rel_err(sim.get_populations()[0], orc.get_populations()) <= 1e-5
    r_g, _ = sim.get_beads()
    r_o, _ = orc.get_beads()
    assert np.abs(r_g - r_o).max() <= 1e-5


def test_fluctuating_equipartition_and_conservation():
    w = small_workload(nx=32, ny=32, nz=32, wall_x=-1, n_beads=0, tau=0.8, lb_kT=LB_KT)
    inp = workloads.build_inputs(w)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    o0 = sim.observables()[0]
    sim.step(200)
    c, wts, _ = oracle.tables()
    acc = np.zeros(4)
    n = 40
    for _ in range(n):
        sim.step(1)
        d = sim.get_deviations()[0].astype(np.float64)
        j = np.tensordot(c.T.astype(float), d, 1)
        acc += [np.mean(j[0] ** 2), np.mean(j[1] ** 2), np.mean(j[2] ** 2), np.mean(d.sum(0) ** 2)]
    acc /= n
    assert np.allclose(acc[:3] / LB_KT, 1.0, atol=0.03), acc[:3] / LB_KT
    assert acc[3] / (3 * LB_KT) == pytest.approx(1.0, abs=0.03)
    o1 = sim.observables()[0]
    assert abs(o1["mass"] - o0["mass"]) < 1e-9 * o0["mass"]
    for a in ("x", "y", "z"):
        assert abs(o1["p_fluid_" + a]) < 1e-4  # 32768 sites of rounding-level momentum


def test_adjoint_refuses_fluctuating_fluid():
    w = small_workload(lb_kT=LB_KT)
    inp = workloads.build_inputs(w)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    with pytest.raises(lbmd.LbmdError):
        sim.adjoint_bytes(4, 2)
