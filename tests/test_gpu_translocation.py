"""Translocation records and per-step radii of gyration (Sec. IV.A, IV.B).

The bead-diagnostics kernel counts the translocated beads of the state each
step starts from, records the radii of gyration of both parts in the step's
diagnostics row and keeps, per realization, the first step at which part of
the chain and all of it had crossed.  The tests hold these to the oracle's
trajectory through exact properties: the radius of gyration of a fixed set of
beads moves by at most the largest bead displacement (it is the RMS distance
from the centroid, a 1-Lipschitz function of the positions), and a bead's side
of the wall can differ between the two runs only where it lies within that
displacement of the threshold x = wall_x + 1/2."""
import numpy as np
import pytest

from gpu_helpers import make_pair, small_workload
from paper_0711_2665_gb300 import lbmd, workloads

pytestmark = pytest.mark.gpu


def _rg(r):
    if len(r) == 0:
        return 0.0
    d = r - r.mean(axis=0)
    return float(np.sqrt((d * d).sum(axis=1).mean()))


def _parts(r, wall_x):
    tr = r[:, 0] > wall_x + 0.5
    return int(tr.sum()), _rg(r[~tr]), _rg(r[tr])


def _first(cond):
    idx = np.flatnonzero(cond)
    return int(idx[0]) if idx.size else -1


# The kernel sums squared distances from a part's centroid as integers of
# 2^-30: each bead adds six rounded terms (half a unit each), so R^2 is off by
# at most 3 * 2^-30 and R by at most 3 * 2^-30 / (2 R) -- 1e-8 covers R > 0.15
# (and R = 0 is exact: a lone bead is its own centroid)
RG_ABS = 1e-8


def test_rows_carry_radii_of_gyration():
    """The row a step records holds the radii of gyration of the state it
    started from, as the two-pass observables compute them."""
    w = small_workload()
    sim, _, _ = make_pair(w)
    sim.step(5)
    for _ in range(3):
        before = sim.observables()[0]
        sim.step(1)
        row = sim.diagnostics(1)[0][-1]
        assert row["n_translocated"] == before["n_translocated"]
        for k in ("rg_untranslocated", "rg_translocated"):
            assert row[k] == pytest.approx(before[k], rel=1e-9, abs=RG_ABS), k


def test_record_follows_the_oracle_trajectory():
    """A 20-bead chain driven through the pore of the 32x16x16 case: the
    record and the per-step rows against the oracle, step by step."""
    w = workloads.get("plain_fp64_small")
    sim, orc, inp = make_pair(w)
    N, wall = int(w["n_beads"]), int(w["wall_x"])
    steps = 220
    g_rows, o_parts, dev, margin = [], [], [], []
    for k in range(steps):
        rg_, _ = sim.get_beads()
        ro, _ = orc.get_beads()
        d = float(np.abs(rg_ - ro).max())
        dev.append(d)
        margin.append(float(np.abs(ro[:, 0] - (wall + 0.5)).min()))
        o_parts.append(_parts(ro, wall))
        g_rows.append(_parts(rg_, wall))
        sim.step(1)
        orc.step(1)
    dev, margin = np.array(dev), np.array(margin)
    rows = sim.diagnostics(steps)[0]
    assert list(rows["step"]) == list(range(steps))
    # the rows against the GPU's own positions: the count exactly, the radii
    # to the fixed-point resolution
    for k in range(steps):
        n, ru, rt = g_rows[k]
        assert rows["n_translocated"][k] == n
        assert rows["rg_untranslocated"][k] == pytest.approx(ru, rel=1e-9, abs=RG_ABS)
        assert rows["rg_translocated"][k] == pytest.approx(rt, rel=1e-9, abs=RG_ABS)
    # the rows against the oracle: the same count wherever no bead lies
    # within the displacement of the threshold; radii within the displacement
    n_o = np.array([p[0] for p in o_parts])
    safe = margin > dev
    assert safe.mean() > 0.9
    assert np.array_equal(rows["n_translocated"][safe], n_o[safe])
    for k in np.flatnonzero(safe):
        for j, key in ((1, "rg_untranslocated"), (2, "rg_translocated")):
            assert abs(rows[key][k] - o_parts[k][j]) <= dev[k] * (1 + 1e-9) + RG_ABS, (k, key)
    # the record: first passages of the rows, and those of the oracle where safe
    rec = sim.translocation()[0]
    t_first = _first(rows["n_translocated"] > 0)
    t_x = _first(rows["n_translocated"] == N)
    assert t_x > 0, "the chain did not translocate within the run"
    assert rec["t_origin"] == 0 and rec["t_first"] == t_first and rec["t_x"] == t_x
    assert rec["max_translocated"] == N
    assert rec["rg_u_origin"] == pytest.approx(o_parts[0][1], rel=1e-9, abs=RG_ABS)
    assert rec["rg_t_x"] == rows["rg_translocated"][t_x]
    for t_g, cond in ((t_first, n_o > 0), (t_x, n_o == N)):
        t_o = _first(cond)
        if safe[min(t_g, t_o)] and safe[max(t_g, t_o)]:
            assert t_g == t_o
        else:
            assert abs(t_g - t_o) <= 2


def _ensemble():
    w = workloads.get("ensemble_fp32", nx=40, ny=20, nz=12, wall_x=20, n_real=3,
                      bead_counts=[6, 14, 0], E=0.1)
    inp = workloads.build_inputs(w)
    return w, inp


def test_ensemble_records_graph_loop_and_reset():
    """Uneven chains (one realization without beads): the records of the graph
    loop equal those of eager steps, each is the first passage of its rows,
    and a reset restarts them at the current step."""
    w, inp = _ensemble()
    eager = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    loop = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    fresh = eager.translocation()
    assert list(fresh["t_origin"]) == [0, 0, 0] and list(fresh["t_x"]) == [-1, -1, -1]
    assert list(fresh["rg_u_origin"]) == [-1.0, -1.0, -1.0]
    n = 300
    eager.step(n)
    loop.step_loop(n)
    a, b = eager.translocation(), loop.translocation()
    assert a.tobytes() == b.tobytes()
    rows = eager.diagnostics(n)
    counts = np.diff(inp["offsets"])
    for r, N in enumerate(counts):
        if N == 0:
            assert a[r]["t_first"] == -1 and a[r]["t_x"] == -1 and a[r]["rg_u_origin"] == -1.0
            continue
        assert a[r]["t_first"] == _first(rows[r]["n_translocated"] > 0)
        assert a[r]["t_x"] == _first(rows[r]["n_translocated"] == N)
        assert a[r]["rg_u_origin"] == rows[r]["rg_untranslocated"][0]
        assert a[r]["max_translocated"] == rows[r]["n_translocated"].max()
    assert (a["t_x"][counts > 0] > 0).all(), "short chains at E = 0.1 translocate within the run"
    # reset: the origin moves to the current step; a chain that is through
    # counts as through at once
    eager.reset_translocation()
    eager.step(4)
    rows = eager.diagnostics(4)
    c = eager.translocation()
    assert list(c["t_origin"]) == [n, n, n]
    for r, N in enumerate(counts):
        if N == 0:
            continue
        assert c[r]["rg_u_origin"] == rows[r]["rg_untranslocated"][0]
        if rows[r]["n_translocated"][0] == N:
            assert c[r]["t_first"] == n and c[r]["t_x"] == n


def test_autotune_keeps_the_records():
    """The autotuner's pseudo-steps run the bead diagnostics as a step does;
    the translocation records, and every diagnostics row a caller can read,
    come out unchanged.  Past the ring's length the slot the pseudo-steps
    write holds the oldest of those rows."""
    w, inp = _ensemble()
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    sim.step(40)
    before = sim.translocation()
    sim.autotune(2)
    assert sim.translocation().tobytes() == before.tobytes()
    sim.step_loop(lbmd.DIAG_RING + 10)
    rows, recs = sim.diagnostics(), sim.translocation()
    assert rows.shape[1] == lbmd.DIAG_RING
    sim.autotune(2)
    assert sim.diagnostics().tobytes() == rows.tobytes()
    assert sim.translocation().tobytes() == recs.tobytes()


def _oracle_tx(w, inp, r, max_steps):
    """First step at whose starting state every bead of realization r has
    unwrapped x > wall_x + 1/2, in the oracle's run (-1 if none)."""
    import oracle
    o0, o1 = int(inp["offsets"][r]), int(inp["offsets"][r + 1])
    orc = oracle.OracleSim(workloads.oracle_params(w, r, o1 - o0), inp["solid"])
    orc.set_beads(inp["r0"][o0:o1])
    thr = w["wall_x"] + 0.5
    for k in range(max_steps + 1):
        if np.all(orc.get_beads()[0][:, 0] > thr):
            return k
        orc.step(1)
    return -1


def test_translocation_time_fp32_and_fp16_against_oracle():
    """Translocation time t_X (Sec. IV.A) of 8 chains of 20 beads in the
    ensemble workload's box (64x32x32, 3x3 pore, E = 0.05, gamma = 0.1,
    k_BT = 1e-4), each with its own start and noise stream, in FP32 and in
    FP16 population storage, against the FP64 oracle run of each chain.
    t_X is a first-passage time of a chaotic trajectory: the runs separate
    through rounding, but the field drives the last beads through the
    threshold at a tenth of a site per step or more, so the times stay within
    a few steps (measured: FP32 at most 2, FP16 at most 1 of t_X = 74..159).
    Bound per chain: max(3, 3% of t_X)."""
    from paper_0711_2665_gb300 import transloc
    got = {}
    for prec in ("fp32", "fp16dev"):
        out = transloc.run([20], 8, 400, chunk=50, overrides={"precision": prec}, autotune=False)
        got[prec] = np.asarray(out["records"]["t_x"])
        w, counts = out["workload"], out["counts"]
    inp = workloads.build_inputs(w)
    want = np.array([_oracle_tx(w, inp, r, 400) for r in range(len(counts))])
    assert np.all(want > 0)
    tol = np.maximum(3, 0.03 * want)
    print("t_X oracle", want.tolist(), {k: v.tolist() for k, v in got.items()})
    for prec, tx in got.items():
        assert np.all(tx > 0), prec
        assert np.all(np.abs(tx - want) <= tol), (prec, tx.tolist(), want.tolist())
