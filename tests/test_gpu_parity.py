"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP32 state, FP32 arithmetic; derivation in the design notes):
  populations after one step      per element, as deviations h = f - w_i:
                                  |h_gpu - h_orc| <= 1e-5 max|h|, plus
                                  (8/6) 1e-5 max|J| within one site of the
                                  corners the beads touch (gpu_helpers)
  bead velocities after one step  <= 1e-5 * max |v| + k 2^-24
  bead positions after one step   <= 1e-5 * max |r(n+1) - r(n)| + 1e-6 + k 2^-24
  coupling u_p and J              <= 1e-5 relative to their max
The floor k 2^-24 is the FP32 bond force: k (|b| - r0) keeps only the
absolute error of |b| ~ 2^-24 r0, and over one LB time unit that force error
moves a bead's velocity (and position) by at most k 2^-24 (6e-6 for k = 100).
The states are developed: a seeded smooth flow of amplitude 1e-2 under the
chain, so that every site's populations deviate from rest.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import (assert_dev_close, deviations, dev_tolerance, developed_pair, load_state, make_pair,
                         near_bead_sites, rel_err, small_workload, to_f32_state)
from paper_0711_2665_gb300 import inputs, lbmd, workloads

pytestmark = pytest.mark.gpu


def _compare_one_step(sim, orc, inp, label="", fp16=False):
    r_before, _ = orc.get_beads()
    sim.step(1)
    orc.step(1)
    h_g = sim.get_deviations()[0]
    h_o = deviations(orc, inp["solid"])
    J_max = 0.0
    near = None
    if orc.n_beads:
        r_g, v_g = sim.get_beads()
        r_o, v_o = orc.get_beads()
        dr = np.abs(r_o - r_before).max()
        floor = orc.params["k_bond"] * 2.0 ** -24
        assert np.abs(r_g - r_o).max() <= 1e-5 * dr + 1e-6 + floor, (label, "r", np.abs(r_g - r_o).max(), dr)
        assert np.abs(v_g - v_o).max() <= 1e-5 * np.abs(v_o).max() + floor, (label, "v", np.abs(v_g - v_o).max())
        up_g, J_g = sim.get_coupling()
        up_o, J_o = orc.last_coupling()
        assert rel_err(up_g, up_o) <= 1e-5 or np.abs(up_g - up_o).max() < 1e-9, (label, "up")
        assert rel_err(J_g, J_o) <= 1e-5, (label, "J", rel_err(J_g, J_o))
        J_max = float(np.abs(J_o).max())
        near = near_bead_sites(r_before, (orc.nx, orc.ny, orc.nz))
    tol = dev_tolerance(h_o, near, J_max, fp16=fp16)
    return assert_dev_close(h_g, h_o, tol, inp["solid"] == 0, label)


def test_rest_state_is_exact_fixed_point():
    w = small_workload(n_beads=0)
    sim, orc, inp = make_pair(w)
    sim.step(5)
    f = sim.get_populations()[0]
    c, wts, _ = oracle.tables()
    fluid = inp["solid"] == 0
    assert np.array_equal(f[:, fluid], np.broadcast_to(wts.astype(np.float32)[:, None], f[:, fluid].shape))
    assert np.all(f[:, ~fluid] == 0)


def test_population_roundtrip_is_exact():
    w = small_workload(n_beads=0)
    sim, orc, inp = make_pair(w)
    rng = np.random.default_rng(1)
    c, wts, _ = oracle.tables()
    f = (wts[:, None, None, None] * (1 + 0.1 * rng.standard_normal((19, w["nz"], w["ny"], w["nx"])))).astype(np.float32)
    f[:, inp["solid"] == 1] = 0
    sim.set_populations(f[None])
    assert np.array_equal(sim.get_populations()[0], f)


def test_one_step_from_developed_state_small():
    w = small_workload()
    sim, orc, inp = developed_pair(w, steps=40)
    for k in range(3):
        _compare_one_step(sim, orc, inp, f"step {k}")


def test_one_step_without_noise_and_with_body_force():
    w = small_workload(kT=0.0, body_force=(1e-5, -2e-6, 0.0), E=0.05, seed=3)
    sim, orc, inp = developed_pair(w, steps=20)
    _compare_one_step(sim, orc, inp)


@pytest.mark.parametrize("name,shape", [
    ("plain_fp64_small", None), ("plain_fp32", None), ("adjoint", None), ("lattice_4m_fp32", None),
    # the particle-kernel shapes the bench's autotuner picks for the 400- and 1000-bead chains
    ("plain_fp32", (8, 16, "pull", "warp")), ("plain_fp32", (4, 16, "pull", "warp")),
    ("plain_fp32", (4, 8, "push", "lanes")), ("lattice_4m_fp32", (2, 16, "pull", "warp")),
])
def test_one_step_at_full_workload_size(name, shape):
    """The named workloads at their full sizes, with the default particle
    shape and with the shapes the bench times: a developed state (a seeded
    flow of amplitude 1e-2 under the chain, two oracle steps), then one step
    on both sides from it, every population compared."""
    w = workloads.get(name, precision="fp32")
    sim, orc, inp = developed_pair(w, steps=2)
    if shape:
        sim.set_md_shape(shape[0], shape[1])
        sim.set_md_exchange(shape[2])
        sim.set_md_bonded(shape[3])
    h0 = deviations(orc, inp["solid"])
    assert np.median(np.abs(h0[:, inp["solid"] == 0])) > 1e-5  # every site carries a flow
    _compare_one_step(sim, orc, inp, name)


def test_first_steps_from_initial_state_c0():
    """Config of the plain FP64 case from its initial state: 30 steps; the
    runs stay within the accumulated FP32 error."""
    w = workloads.get("plain_fp64_small")
    sim, orc, inp = make_pair(w)
    for k in range(3):
        sim.step(10)
        orc.step(10)
        f_g = sim.get_populations()[0]
        f_o = orc.get_populations()
        assert rel_err(f_g, f_o) < 1e-4 * (k + 1), rel_err(f_g, f_o)
        r_g, _ = sim.get_beads()
        r_o, _ = orc.get_beads()
        assert np.abs(r_g - r_o).max() < 1e-3


def test_observables_match_oracle():
    w = small_workload()
    sim, orc, inp = make_pair(w)
    orc.step(25)
    f32, r, v = to_f32_state(orc)
    load_state(sim, orc, f32, r, v, 25)
    og = sim.observables()[0]
    oo = orc.observables()
    assert og["status"] == 0 and og["step"] == 25
    assert og["mass"] == pytest.approx(oo["mass"], rel=1e-9)
    for k in ("p_fluid_x", "p_fluid_y", "p_fluid_z", "p_beads_x", "p_beads_y", "p_beads_z"):
        assert og[k] == pytest.approx(oo[k], rel=1e-5, abs=1e-8), k
    for k in ("com_x", "com_y", "com_z", "rg_untranslocated", "rg_translocated"):
        assert og[k] == pytest.approx(oo[k], rel=1e-6, abs=1e-6), k
    assert og["n_translocated"] == oo["n_translocated"]
    for k in ("dWH_dt", "dWE_dt"):
        assert og[k] == pytest.approx(oo[k], rel=1e-4, abs=1e-9), k


def test_per_step_diagnostics_match_observables():
    """The row each step records (fluid sums from the stream-collide kernel,
    bead sums from the bead-diagnostics kernel) equals the observables of the
    state the step started from."""
    w = small_workload()
    sim, orc, inp = make_pair(w)
    sim.step(7)
    before = sim.observables()[0]
    sim.step(1)
    row = sim.diagnostics(4)[0][-1]
    assert row["step"] == 7
    assert row["mass"] == pytest.approx(before["mass"], rel=1e-10)
    for a, k in enumerate("xyz"):
        assert row["p_fluid"][a] == pytest.approx(before[f"p_fluid_{k}"], rel=1e-5, abs=1e-9)
        assert row["p_beads"][a] == pytest.approx(before[f"p_beads_{k}"], rel=1e-6, abs=1e-12)
        assert row["com"][a] == pytest.approx(before[f"com_{k}"], rel=1e-7)
    assert row["dWH_dt"] == pytest.approx(before["dWH_dt"], rel=1e-4, abs=1e-10)


def test_graph_eager_and_tiles_are_bit_identical():
    w = small_workload()
    runs = []
    for mode in ("eager", "graph", "tiles"):
        sim, orc, inp = make_pair(w)
        if mode == "graph":
            sim.set_graph(4)
        if mode == "tiles":
            sim.set_tiles(2, 3)
        sim.step(10)
        runs.append((sim.get_populations(), *sim.get_beads()))
    for other in runs[1:]:
        for a, b in zip(runs[0], other):
            assert np.array_equal(a, b)


def test_autotune_keeps_results():
    """The autotuner (tiles, then particle-kernel shape) leaves the state as it
    found it, and a run with the tuned shapes equals a run given the same
    shapes explicitly, bit for bit; a shape fixed by the caller is kept."""
    w = small_workload()
    sim, orc, inp = make_pair(w)
    sim.step(3)
    before = (sim.get_deviations(), *sim.get_beads(), sim.step_count)
    by, zc = sim.autotune(2)
    after = (sim.get_deviations(), *sim.get_beads(), sim.step_count)
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    assert (by, zc) == sim.tiles()
    shape = sim.md_shape()
    sim.step(3)
    sim2, _, _ = make_pair(w)
    sim2.set_tiles(by, zc)
    sim2.set_md_shape(*shape)
    sim2.step(6)
    assert np.array_equal(sim.get_populations(), sim2.get_populations())
    sim2.autotune(2)
    assert sim2.md_shape() == shape


def test_reserving_sms_changes_nothing_and_is_kept():
    """The particle blocks claiming their SMs' shared memory (or not) changes
    where the kernels run, not what they compute: both give the same state
    bit for bit; a choice fixed by the caller survives the autotuner, and
    "auto" hands it back."""
    w = small_workload()
    inp = workloads.build_inputs(w)
    out = []
    for mode in ("share", "reserve"):
        sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
        sim.set_md_reserve(mode)
        assert sim.md_reserve() == (mode == "reserve")
        sim.step(6)
        out.append((sim.get_deviations(), *sim.get_beads()))
        sim.autotune(1)
        assert sim.md_reserve() == (mode == "reserve")
        sim.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    sim.set_md_reserve("reserve")
    sim.set_md_reserve("auto")
    sim.autotune(1)  # free again: either choice is valid
    assert sim.md_reserve() in (True, False)
    with pytest.raises(KeyError):
        sim.set_md_reserve("always")


def test_ensemble_realizations_match_oracle():
    """Three realizations with chains of different lengths in one launch; each
    matches its own oracle run (realization index in the Philox key)."""
    w = small_workload(n_real=3, n_beads=(10, 30), chain_seed=11)
    inp = workloads.build_inputs(w)
    assert len(set(inp["counts"].tolist())) > 1
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    sim.step(4)
    f_all = sim.get_populations()
    r_all, v_all = sim.get_beads()
    for r in range(3):
        o0, o1 = inp["offsets"][r], inp["offsets"][r + 1]
        orc = oracle.OracleSim(workloads.oracle_params(w, r, o1 - o0), inp["solid"])
        orc.set_beads(inp["r0"][o0:o1])
        orc.step(4)
        assert rel_err(f_all[r], orc.get_populations()) < 1e-5
        ro, vo = orc.get_beads()
        assert np.abs(r_all[o0:o1] - ro).max() < 1e-5
        assert np.abs(v_all[o0:o1] - vo).max() < 1e-5 * np.abs(vo).max() + 4 * w["k_bond"] * 2.0 ** -24


def test_nonfinite_state_is_reported():
    """A NaN planted in the populations (host-side fault injection) is caught
    by the step's diagnostics and reported by lbmd_check."""
    w = small_workload()
    sim, orc, inp = make_pair(w)
    f = sim.get_populations()
    f[0, 3, 5, 7, 9] = np.nan
    sim.set_populations(f)
    sim.step(2)
    with pytest.raises(lbmd.LbmdError) as e:
        sim.check()
    assert e.value.status == 3


def test_cluster_size_does_not_change_the_arithmetic():
    """With the lanes per bead and the bonded mode fixed, spreading a chain
    over 1, 2, 4, 8 or 16 blocks of a cluster changes who computes a bead,
    not how: every run of 40 steps (list rebuilds included) ends in the same
    state bit for bit.  Other lane counts split each pair sum differently, and
    the two bonded modes add the bonded terms in different orders: after one
    step they agree to rounding.  Over many steps they part: the pore field is
    a step function of position, so a rounding difference can decide a kick
    of E h."""
    w = small_workload(n_beads=48, chain_seed=11)
    inp = workloads.build_inputs(w)

    def run(T, C, n, bonded="lanes"):
        sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
        sim.set_md_shape(T, C)
        sim.set_md_bonded(bonded)
        assert sim.md_bonded() == bonded
        sim.step(n)
        sim.check()
        out = (sim.get_deviations(), *sim.get_beads())
        sim.close()
        return out

    for bonded in ("lanes", "warp"):
        ref = run(4, 1, 40, bonded)
        for C in (2, 4, 8, 16):
            for a, b in zip(ref, run(4, C, 40, bonded)):
                assert np.array_equal(a, b), (bonded, C)
    one = run(4, 1, 1)
    floor = w["k_bond"] * 2.0 ** -24
    for T, C, bonded in ((2, 4, "lanes"), (8, 2, "lanes"), (1, 1, "lanes"), (4, 1, "warp"), (8, 16, "warp")):
        other = run(T, C, 1, bonded)
        assert np.abs(other[1] - one[1]).max() <= 1e-6 + floor, (T, C, bonded)
        assert np.abs(other[2] - one[2]).max() <= 1e-5 * np.abs(one[2]).max() + floor, (T, C, bonded)


def _run_exchange(w, inp, v0, mode, shape, n):
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    sim.set_beads(inp["r0"], v0)
    sim.set_md_shape(*shape)
    sim.set_md_exchange(mode)
    assert sim.md_exchange() == mode
    sim.profile(True)
    sim.step(n)
    rebuilds = sim.kernel_times()["particles.rebuilds"][0]
    sim.profile(False)
    sim.check()
    out = (sim.get_deviations(), *sim.get_beads(), *sim.get_coupling())
    sim.close()
    return out, rebuilds


@pytest.mark.parametrize("case", ["chain over 8 blocks", "chain over 16 blocks", "hashed lists", "shared clusters"])
def test_exchange_modes_are_bit_identical(case):
    """Push (every block's replica written) and pull (each block copies the
    beads its force terms read, the whole chain at a list rebuild) move the
    same positions between a chain's blocks: runs that rebuild their lists end
    in the same state bit for bit.  The cases cover a chain spread over a
    cluster of 8 and of 16, a chain above 512 beads (cell-hash lists) and
    uneven chains that share clusters (some of one block, which exchange
    nothing).  The beads start with velocities of 0.1 per component, so that
    they cross the half skin within the run."""
    if case == "chain over 8 blocks":
        w, shape = small_workload(n_beads=48, chain_seed=11), (4, 8)
    elif case == "chain over 16 blocks":
        w, shape = small_workload(nx=48, ny=32, nz=32, wall_x=24, n_beads=160, chain_seed=5), (2, 16)
    elif case == "hashed lists":
        w, shape = workloads.get("plain_fp32", nx=64, ny=48, nz=48, wall_x=40, n_beads=600), (4, 8)
    else:
        w, shape = small_workload(n_real=5, bead_counts=[40, 6, 25, 12, 33], chain_seed=3), (4, 4)
    inp = workloads.build_inputs(w)
    v0 = 0.1 * np.random.default_rng(4).choice([-1.0, 1.0], size=inp["r0"].shape)
    push, _ = _run_exchange(w, inp, v0, "push", shape, 30)
    pull, rebuilds = _run_exchange(w, inp, v0, "pull", shape, 30)
    assert rebuilds > 0, "no list rebuild: the whole-chain copy was not exercised"
    for a, b in zip(push, pull):
        assert np.array_equal(a, b), case
