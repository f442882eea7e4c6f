"""Reverse mode on the GPU (lbmd_adjoint) against the FP64 oracle.

* Parity with the oracle's discrete adjoint on a small coupled case (wall,
  pore, noise, a chain partly inside the pore channel, ragged x tiles,
  ragged checkpoint segments): loss, dL/dgamma, dL/dE and every dL/dr0.
  Tolerances: the GPU differentiates its FP32 step, the oracle its FP64 step;
  the two trajectories agree to ~1e-6 relative (see the forward parity
  tests), the FP32 adjoint sums over K * M * M^b sub-steps carry relative
  errors of order 1e-5, so the gradients are compared at 1e-3 relative (and
  the coordinates at 1e-3 of the largest coordinate gradient).
* The checkpoint interval changes nothing: gradients are bit-identical for
  every interval (the replays repeat the forward bit for bit).
* The handle ends in the state K forward steps reach.
* Realizations of an ensemble are independent: each one's gradient equals the
  gradient of the same chain run alone (same MD launch shape).
* The autograd wrapper returns the adjoint's gradients scaled by the incoming
  gradient.
* On the full adjoint workload (96x48x48, N = 100) at K = 30 (checkpoint
  segments 20 + 10) the gradient matches the oracle adjoint entry by entry and
  FP64 central differences (h = 1e-4, pore-field events held) for gamma, E
  and sampled coordinates; the K = 200 run with checkpoints every 20 replays
  the forward exactly (see the note above the full-workload tests for why the
  gradient values are not compared there).
"""
import multiprocessing as mp

import numpy as np
import pytest

import oracle
from gpu_helpers import small_workload
from paper_0711_2665_gb300 import lbmd, workloads

pytestmark = pytest.mark.gpu


def _case(K=8, n_beads=10, **kw):
    w = small_workload(nx=40, ny=20, nz=12, wall_x=20, n_beads=n_beads, kappa_bend=1e-3, **kw)
    inp = workloads.build_inputs(w)
    r0 = inp["r0"].copy()
    # the first bead (at the pore entrance, on lattice sites) moves into the
    # pore channel and off the cell faces, where the weights have kinks
    r0[0] += (0.4, 0.137, 0.137)
    inp["r0"] = r0
    return w, inp


def _gpu(w, inp, K, C, shape=None):
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    if shape:
        sim.set_md_shape(*shape)
    g = sim.adjoint(K, C)
    return sim, g


def test_adjoint_matches_oracle_adjoint():
    K = 8
    w, inp = _case(K)
    sim, g = _gpu(w, inp, K, 3)
    o = oracle.adjoint(workloads.oracle_params(w, 0, inp["r0"].shape[0]), inp["solid"], inp["r0"], K)
    # FP32 bond forces carry an absolute error k 2^-24 per unit time (see the
    # forward parity tests); over K steps the chain's mean moves by up to K times that
    assert abs(g["loss"][0] - o["loss"]) <= K * w["k_bond"] * 2.0 ** -24 + 1e-5 * abs(o["loss"])
    assert g["dgamma"][0] == pytest.approx(o["dgamma"], rel=1e-3)
    assert g["dE"][0] == pytest.approx(o["dE"], rel=1e-3)
    scale = np.abs(o["dr0"]).max()
    err = np.abs(g["dr0"] - o["dr0"])
    assert np.all(err <= 1e-3 * scale + 1e-3 * np.abs(o["dr0"])), (err.max(), scale)


def test_checkpoint_interval_and_final_state():
    K = 7
    w, inp = _case(K)
    sims = []
    res = []
    for C in (1, 3, 7, 20):
        sim, g = _gpu(w, inp, K, C)
        sims.append(sim)
        res.append(g)
    for g in res[1:]:
        assert np.array_equal(g["dr0"], res[0]["dr0"])
        assert g["dgamma"][0] == res[0]["dgamma"][0] and g["dE"][0] == res[0]["dE"][0]
        assert g["loss"][0] == res[0]["loss"][0]
    ref = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    ref.step(K)
    for sim in sims:
        assert sim.step_count == K
        assert np.array_equal(sim.get_deviations(), ref.get_deviations())
        ra, va = sim.get_beads()
        rb, vb = ref.get_beads()
        assert np.array_equal(ra, rb) and np.array_equal(va, vb)


def test_ensemble_realizations_are_independent():
    K = 5
    w1, inp1 = _case(K, n_beads=9)
    w2, inp2 = _case(K, n_beads=6, seed=11, chain_seed=11)
    # one handle with both chains; realization r draws its noise with key
    # (seed, r), so chain 1 is compared with a one-realization run (r = 0) and
    # chain 2 with the oracle at realization index 1
    we = dict(w1)
    we["n_real"] = 2
    solid = inp1["solid"]
    offs = np.array([0, 9, 15], dtype=np.int32)
    r0 = np.concatenate([inp1["r0"], inp2["r0"]])
    sim = lbmd.Simulation(we, solid, offs, r0)
    sim.set_md_shape(2, 1)
    ge = sim.adjoint(K, 2)
    s1 = lbmd.Simulation(w1, solid, np.array([0, 9], dtype=np.int32), inp1["r0"])
    s1.set_md_shape(2, 1)
    g1 = s1.adjoint(K, 2)
    assert np.array_equal(ge["dr0"][:9], g1["dr0"])
    assert ge["dgamma"][0] == g1["dgamma"][0] and ge["dE"][0] == g1["dE"][0]
    # realization 1 against the oracle (its noise key uses realization 1)
    o = oracle.adjoint(workloads.oracle_params(we, 1, 6), solid, inp2["r0"], K)
    assert ge["dgamma"][1] == pytest.approx(o["dgamma"], rel=1e-3)
    scale = np.abs(o["dr0"]).max()
    assert np.all(np.abs(ge["dr0"][9:] - o["dr0"]) <= 1e-3 * scale + 1e-3 * np.abs(o["dr0"]))


def test_autograd_function():
    import torch
    K = 4
    w, inp = _case(K)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    r0 = torch.tensor(inp["r0"], dtype=torch.float64, requires_grad=True)
    gam = torch.tensor(w["gamma"], dtype=torch.float64, requires_grad=True)
    E = torch.tensor(w["E"], dtype=torch.float64, requires_grad=True)
    L = lbmd.com_displacement(sim, r0, gam, E, K, checkpoint_every=2)
    (2.5 * L.sum()).backward()
    sim2 = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    g = sim2.adjoint(K, 2)
    assert float(L[0]) == g["loss"][0]
    assert np.allclose(r0.grad.numpy(), 2.5 * g["dr0"], rtol=0, atol=0)
    assert float(gam.grad) == 2.5 * g["dgamma"][0]
    assert float(E.grad) == 2.5 * g["dE"][0]


# ---------------------------------------------------------------------------
# the full adjoint workload (96x48x48 lattice, wall with a 4x4 pore, N = 100)
# ---------------------------------------------------------------------------
# The chain dynamics of this workload is chaotic: the exact derivative of the
# discrete step grows about 20-fold every 20 LB steps (oracle adjoint norm 33
# at K = 30, 645 at K = 50, ~1e19 at K = 200), and central differences with
# the field events held agree with it only inside that predictability window
# (h = 1e-8: to 1e-5 at K = 30 and 5e-4 at K = 50; no h resolves K = 200).  The
# gradients are therefore checked on the full workload at K = 30 (checkpoint
# segments of 20 and 10 steps); the K = 200 run with checkpoints every 20 is
# checked for its replay (final state, loss) and finiteness.
def _fd_run(args):
    params, solid, r0, K, trace = args
    s = oracle.OracleSim(params, solid)
    s.set_beads(r0)
    if trace is not None:
        s.channel_trace(2, trace)
    x0 = r0[:, 0].mean()
    s.step(K)
    return s.get_beads()[0][:, 0].mean() - x0, s.event_counts()


def _full_case():
    w = workloads.get("adjoint")
    inp = workloads.build_inputs(w)
    r0 = inp["r0"].copy()
    r0[0, 1:] += 0.137  # the first bead off the cell faces, where the weights have kinks
    return w, inp, r0


@pytest.mark.slow
def test_full_workload_against_finite_differences():
    w, inp, r0 = _full_case()
    K, C, h = 30, w["checkpoint_every"], 1e-4
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], r0)
    g = sim.adjoint(K, C)
    P = workloads.oracle_params(w, 0, r0.shape[0])
    # FP64 oracle: its adjoint, and central differences with the pore-field
    # events of the unperturbed run held (the field is a step function of the
    # position; plain differences at h = 1e-4 already cross a few kicks)
    o = oracle.adjoint(P, inp["solid"], r0, K)
    base = oracle.OracleSim(P, inp["solid"])
    base.set_beads(r0)
    trace = np.zeros(K * 2 * w["md_outer"] * r0.shape[0], dtype=np.int32)
    base.channel_trace(1, trace)
    base.step(K)
    rng = np.random.default_rng(0)
    coords = [(0, 0), (r0.shape[0] // 2, 1), (r0.shape[0] - 1, 2)] + \
             [(int(i), int(a)) for i, a in zip(rng.integers(0, r0.shape[0], 5), rng.integers(0, 3, 5))]
    jobs = []
    for name in ("gamma", "E"):
        for sgn in (1, -1):
            Pq = dict(P)
            Pq[name] += sgn * h
            jobs.append((Pq, inp["solid"], r0, K, trace))
    for i, a in coords:
        for sgn in (1, -1):
            rq = r0.copy()
            rq[i, a] += sgn * h
            jobs.append((P, inp["solid"], rq, K, trace))
    with mp.get_context("spawn").Pool(min(len(jobs), max(1, mp.cpu_count()))) as pool:
        out = pool.map(_fd_run, jobs)
    fd = [(out[2 * k][0] - out[2 * k + 1][0]) / (2 * h) for k in range(len(out) // 2)]
    # against the oracle adjoint, every entry.  The FP32 and FP64 trajectories
    # part by rounding, and the chaotic growth that enlarges the gradient
    # (its largest entry grows ~20-fold from K = 5 to K = 30) enlarges that
    # parting too: agreement is 1e-6 at K = 5 and ~1e-3 at K = 30 (measured),
    # so the bound here is 3e-3 (gamma, E) and 1e-2 of the largest entry (r0)
    assert abs(g["loss"][0] - o["loss"]) <= K * w["k_bond"] * 2.0 ** -24 + 1e-5 * abs(o["loss"])
    assert g["dgamma"][0] == pytest.approx(o["dgamma"], rel=3e-3)
    assert g["dE"][0] == pytest.approx(o["dE"], rel=3e-3)
    scale = np.abs(o["dr0"]).max()
    assert np.all(np.abs(g["dr0"] - o["dr0"]) <= 1e-2 * scale)
    # against FP64 central differences (h = 1e-4): the difference quotient
    # itself is off by O(h) (kinks of the weights) and O(h^2) terms the chaotic
    # growth enlarges; at K = 30 that is below 1.5e-3 for gamma and E
    assert g["dgamma"][0] == pytest.approx(fd[0], rel=3e-3)
    assert g["dE"][0] == pytest.approx(fd[1], rel=3e-3)
    norm = np.linalg.norm(g["dr0"])
    for (i, a), fdv in zip(coords, fd[2:]):
        assert abs(g["dr0"][i, a] - fdv) <= 1e-2 * norm, (i, a, g["dr0"][i, a], fdv, norm)


@pytest.mark.slow
def test_full_workload_200_steps_replay():
    w, inp, r0 = _full_case()
    K, C = w["steps"], w["checkpoint_every"]
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], r0)
    g = sim.adjoint(K, C)
    ref = lbmd.Simulation(w, inp["solid"], inp["offsets"], r0)
    ref.step(K)
    assert sim.step_count == K
    assert np.array_equal(sim.get_deviations(), ref.get_deviations())
    ra, _ = sim.get_beads()
    rb, _ = ref.get_beads()
    assert np.array_equal(ra, rb)
    assert g["loss"][0] == pytest.approx(rb[:, 0].mean() - r0[:, 0].mean(), rel=1e-12)
    assert np.all(np.isfinite(g["dr0"])) and np.isfinite(g["dgamma"][0]) and np.isfinite(g["dE"][0])
