"""Edge cases of the CUDA path against the FP64 oracle: the FP16 and ensemble
workloads at their full sizes, the longest chain one realization may hold
(1024 beads), degenerate physics (no friction or noise, no field, no wall,
the narrowest and a closed pore) and an ensemble member without beads.

Tolerances are those of the parity tests, on the deviations h = f - w_i
element by element (gpu_helpers: FP32 rounding, the coupling term near the
beads, and for FP16 storage half an FP16 ulp of each element, 2^-11 |h|, or
2^-37 below the FP16 normal range); k 2^-24 bond-force floor for the beads."""
import numpy as np
import pytest

import oracle
from gpu_helpers import (assert_dev_close, deviations, dev_tolerance, developed_pair, load_dev_state, make_pair,
                         near_bead_sites, small_workload)
from paper_0711_2665_gb300 import inputs as inp_mod
from paper_0711_2665_gb300 import lbmd, workloads

pytestmark = pytest.mark.gpu


def _one_step(sim, orc, inp, label, fp16=False):
    r_before, _ = orc.get_beads()
    sim.step(1)
    orc.step(1)
    h_g = sim.get_deviations()[0]
    h_o = deviations(orc, inp["solid"])
    near, J_max = None, 0.0
    if orc.n_beads:
        r_g, v_g = sim.get_beads()
        r_o, v_o = orc.get_beads()
        floor = orc.params["k_bond"] * 2.0 ** -24
        dr = np.abs(r_o - r_before).max()
        assert np.abs(r_g - r_o).max() <= 1e-5 * dr + 1e-6 + floor, (label, "r")
        assert np.abs(v_g - v_o).max() <= 1e-5 * np.abs(v_o).max() + floor, (label, "v")
        J_max = float(np.abs(orc.last_coupling()[1]).max())
        near = near_bead_sites(r_before, (orc.nx, orc.ny, orc.nz))
    return assert_dev_close(h_g, h_o, dev_tolerance(h_o, near, J_max, fp16), inp["solid"] == 0, label)


def _developed_pair(w, steps=3):
    return developed_pair(w, steps=steps)


def test_longest_chain_1024_beads():
    w = workloads.get("plain_fp32", n_beads=1024)
    sim, orc, inp = _developed_pair(w, 2)
    _one_step(sim, orc, inp, "N=1024")


@pytest.mark.parametrize("label,kw", [
    ("no friction or noise", dict(gamma=0.0, kT=0.0)),
    ("no field", dict(E=0.0)),
    ("no wall", dict(wall_x=-1)),
    ("1x1 pore", dict(pore_h=1)),
    ("closed wall", dict(pore_h=0)),
])
def test_degenerate_physics(label, kw):
    w = small_workload(**kw)
    sim, orc, inp = _developed_pair(w, 5)
    _one_step(sim, orc, inp, label)
    if kw.get("gamma") == 0.0:
        # the beads never touch the fluid
        up, J = sim.get_coupling()
        assert np.all(J == 0.0)


def test_ensemble_member_without_beads():
    w = small_workload(n_real=3, bead_counts=[12, 0, 9], chain_seed=5)
    inp = workloads.build_inputs(w)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    sim.step(4)
    h_all = sim.get_deviations()
    r_all, _ = sim.get_beads()
    for r in range(3):
        o0, o1 = int(inp["offsets"][r]), int(inp["offsets"][r + 1])
        orc = oracle.OracleSim(workloads.oracle_params(w, r, o1 - o0), inp["solid"])
        if o1 > o0:
            orc.set_beads(inp["r0"][o0:o1])
        orc.step(4)
        h_o = deviations(orc, inp["solid"])
        dims = (w["nx"], w["ny"], w["nz"])
        # four steps: four times the one-step bound; the chain moves less than
        # a site, so the coupling's sites lie within 2 of its cells
        near = near_bead_sites(inp["r0"][o0:o1], dims, pad=1) if o1 > o0 else None
        J_max = float(np.abs(orc.last_coupling()[1]).max()) if o1 > o0 else 0.0
        assert_dev_close(h_all[r], h_o, 4.0 * dev_tolerance(h_o, near, J_max), inp["solid"] == 0, r)
        if o1 > o0:
            assert np.abs(r_all[o0:o1] - orc.get_beads()[0]).max() < 1e-5
    obs = sim.observables()
    assert obs[1]["p_beads_x"] == obs[1]["p_beads_y"] == obs[1]["p_beads_z"] == 0.0
    assert obs[1]["n_translocated"] == 0.0
    sim.check()


def test_ensemble_full_size_sampled_realizations():
    """64 x 64x32x32 with chains of 20..200 beads, each realization under its
    own seeded flow of amplitude 1e-2, in the step-loop launch the bench
    times: four steps, then realizations 0, 31 and 63 against the oracle
    (over four steps the FP32 bound of one step applies four times)."""
    w = workloads.get("ensemble_fp32")
    inp = workloads.build_inputs(w)
    dims = (w["nx"], w["ny"], w["nz"])
    u = np.stack([inp_mod.smooth_random_velocity(*dims, 1e-2, 1000 + r) for r in range(w["n_real"])])
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    sim.autotune(2)
    sim.init_fluid(None, u)
    sim.step_loop(4)
    h_all = sim.get_deviations()
    r_all, v_all = sim.get_beads()
    for r in (0, 31, 63):
        o0, o1 = int(inp["offsets"][r]), int(inp["offsets"][r + 1])
        orc = oracle.OracleSim(workloads.oracle_params(w, r, o1 - o0), inp["solid"])
        orc.set_beads(inp["r0"][o0:o1])
        orc.init_fluid(None, u[r])
        orc.step(4)
        h_o = deviations(orc, inp["solid"])
        J_max = float(np.abs(orc.last_coupling()[1]).max())
        # the chain moves less than a site in four steps: the coupling's
        # sites lie within 2 of its starting cells
        near = near_bead_sites(inp["r0"][o0:o1], dims, pad=1)
        tol = 4.0 * dev_tolerance(h_o, near, J_max)
        assert_dev_close(h_all[r], h_o, tol, inp["solid"] == 0, r)
        ro, vo = orc.get_beads()
        assert np.abs(r_all[o0:o1] - ro).max() < 1e-5, r
        assert np.abs(v_all[o0:o1] - vo).max() < 1e-5 * np.abs(vo).max() + 4 * w["k_bond"] * 2.0 ** -24, r


def _fp16_state(orc, solid):
    """The oracle's state rounded to what FP16 storage holds: h 2^12 to the
    nearest FP16 value (numpy's IEEE round to nearest even), back in FP32."""
    h = deviations(orc, solid)
    return ((h * 4096.0).astype(np.float16).astype(np.float32) / np.float32(4096.0)).astype(np.float32)


@pytest.mark.parametrize("shape", [None, (4, 16, "pull", "warp")])
def test_fp16dev_full_size_one_step(shape):
    """256x128x128 with FP16 deviations and a 1000-bead chain under a seeded
    flow of amplitude 1e-2: one step from the same FP16-representable state
    stays within FP16 storage rounding element by element, with the default
    particle shape and with the one the bench's autotuner picks."""
    w = workloads.get("fp16dev")
    sim, orc, inp = make_pair(w)
    if shape:
        sim.set_md_shape(shape[0], shape[1])
        sim.set_md_exchange(shape[2])
        sim.set_md_bonded(shape[3])
    orc.init_fluid(None, inp_mod.smooth_random_velocity(w["nx"], w["ny"], w["nz"], 1e-2, 11))
    orc.step(2)
    r, v = orc.get_beads()
    load_dev_state(sim, orc, _fp16_state(orc, inp["solid"]), r.copy(), v.astype(np.float32).astype(np.float64),
                   2, inp["solid"])
    _one_step(sim, orc, inp, "fp16dev", fp16=True)
