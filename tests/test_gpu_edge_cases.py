"""Edge cases of the CUDA path against the FP64 oracle: the FP16 and ensemble
workloads at their full sizes, the longest chain one realization may hold
(1024 beads), degenerate physics (no friction or noise, no field, no wall,
the narrowest and a closed pore) and an ensemble member without beads.

Tolerances are those of the parity tests (FP32 rounding; k 2^-24 bond-force
floor for the beads); FP16 storage adds half an FP16 ulp of the largest
deviation (2^-11 relative)."""
import numpy as np
import pytest

import oracle
from gpu_helpers import load_state, make_pair, rel_err, small_workload, to_f32_state
from paper_0711_2665_gb300 import lbmd, workloads

pytestmark = pytest.mark.gpu


def _one_step(sim, orc, label, pop_tol=1e-5):
    r_before, _ = orc.get_beads()
    sim.step(1)
    orc.step(1)
    ef = rel_err(sim.get_populations()[0], orc.get_populations())
    assert ef <= pop_tol, (label, "populations", ef)
    if orc.n_beads:
        r_g, v_g = sim.get_beads()
        r_o, v_o = orc.get_beads()
        floor = orc.params["k_bond"] * 2.0 ** -24
        dr = np.abs(r_o - r_before).max()
        assert np.abs(r_g - r_o).max() <= 1e-5 * dr + 1e-6 + floor, (label, "r")
        assert np.abs(v_g - v_o).max() <= 1e-5 * np.abs(v_o).max() + floor, (label, "v")


def _developed_pair(w, steps=3):
    sim, orc, inp = make_pair(w)
    orc.step(steps)
    f32, r, v = to_f32_state(orc)
    load_state(sim, orc, f32, r, v, steps)
    return sim, orc, inp


def test_longest_chain_1024_beads():
    w = workloads.get("plain_fp32", n_beads=1024)
    sim, orc, inp = _developed_pair(w, 2)
    _one_step(sim, orc, "N=1024")


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
    _one_step(sim, orc, label)
    if kw.get("gamma") == 0.0:
        # the beads never touch the fluid: it stays at rest (up to the FP32
        # rounding of the weights in the state loaded from the oracle)
        f = sim.get_populations()[0]
        _, wts, _ = oracle.tables()
        fluid = inp["solid"] == 0
        assert np.abs(f[:, fluid] - wts[:, None]).max() < 1e-7
        up, J = sim.get_coupling()
        assert np.all(J == 0.0)


def test_ensemble_member_without_beads():
    w = small_workload(n_real=3, bead_counts=[12, 0, 9], chain_seed=5)
    inp = workloads.build_inputs(w)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    sim.step(4)
    f_all = sim.get_populations()
    r_all, _ = sim.get_beads()
    for r in range(3):
        o0, o1 = int(inp["offsets"][r]), int(inp["offsets"][r + 1])
        orc = oracle.OracleSim(workloads.oracle_params(w, r, o1 - o0), inp["solid"])
        if o1 > o0:
            orc.set_beads(inp["r0"][o0:o1])
        orc.step(4)
        assert rel_err(f_all[r], orc.get_populations()) < 1e-5, r
        if o1 > o0:
            assert np.abs(r_all[o0:o1] - orc.get_beads()[0]).max() < 1e-5
    obs = sim.observables()
    assert obs[1]["p_beads_x"] == obs[1]["p_beads_y"] == obs[1]["p_beads_z"] == 0.0
    assert obs[1]["n_translocated"] == 0.0
    sim.check()


def test_ensemble_full_size_sampled_realizations():
    """64 x 64x32x32 with chains of 20..200 beads, in the step-loop launch the
    bench times: four steps, then realizations 0, 31 and 63 against the oracle."""
    w = workloads.get("ensemble_fp32")
    inp = workloads.build_inputs(w)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    sim.autotune(2)
    sim.step_loop(4)
    f_all = sim.get_populations()
    r_all, v_all = sim.get_beads()
    for r in (0, 31, 63):
        o0, o1 = int(inp["offsets"][r]), int(inp["offsets"][r + 1])
        orc = oracle.OracleSim(workloads.oracle_params(w, r, o1 - o0), inp["solid"])
        orc.set_beads(inp["r0"][o0:o1])
        orc.step(4)
        assert rel_err(f_all[r], orc.get_populations()) < 1e-5, r
        ro, vo = orc.get_beads()
        assert np.abs(r_all[o0:o1] - ro).max() < 1e-5, r
        assert np.abs(v_all[o0:o1] - vo).max() < 1e-5 * np.abs(vo).max() + 4 * w["k_bond"] * 2.0 ** -24, r


@pytest.mark.parametrize("shape", [None, (4, 16, "pull", "warp")])
def test_fp16dev_full_size_one_step(shape):
    """256x128x128 with FP16 deviations and a 1000-bead chain: one step from the
    same FP16-representable state stays within the storage rounding, with the
    default particle shape and with the one the bench's autotuner picks."""
    w = workloads.get("fp16dev")
    sim, orc, inp = make_pair(w)
    if shape:
        sim.set_md_shape(shape[0], shape[1])
        sim.set_md_exchange(shape[2])
        sim.set_md_bonded(shape[3])
    orc.step(2)
    f32, r, v = to_f32_state(orc)
    _, wts, _ = oracle.tables()
    fluid = inp["solid"] == 0
    wb = wts[:, None, None, None].astype(np.float32)
    f16 = ((f32 - wb) * 4096.0).astype(np.float16).astype(np.float32) / 4096.0 + wb
    f16[:, ~fluid] = 0
    load_state(sim, orc, f16.astype(np.float32), r, v, 2)
    sim.step(1)
    orc.step(1)
    fo = orc.get_populations()
    fg = sim.get_populations()[0]
    devmax = np.abs(fo - wts[:, None, None, None])[:, fluid].max()
    assert np.abs(fg - fo)[:, fluid].max() <= 2.0 ** -11 * devmax + 1e-6
