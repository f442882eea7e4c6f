"""Shared helpers of the GPU tests: build a CUDA-path Simulation and an oracle
run of the same workload from the same seeded inputs, move one state into
both, and compare populations as deviations h = f - w_i.

Population tolerance (one step from one shared state, element by element):

  |h_gpu - h_orc| <= 1e-5 max|h_orc| + 1e-15             FP32 arithmetic
                   + 2^-11 |h_orc| + 2^-37                 FP16 storage only
                   + (8/6) 1e-5 max|J_orc|                 sites the beads touch
                   + 2^-11 |h_orc|                         ... with FP16 storage

FP32: the library stores h itself, so a step's rounding is relative to the
deviations, not to w_i (a few 1e-7 of max|h| for the 19-term moment sums).
FP16 storage keeps h 2^12 with 11 significant bits: a stored value is within
half an ulp, 2^-11 |h|, of the FP32 result, or within 2^-25 2^-12 = 2^-37
where h 2^12 falls below the smallest normal FP16 number.  The beads hand
their impulse J to the fluid as the source S_i = 3 w_i c_i.G, G = -sum_p W_p
J_p over the corners of each bead's cell: |dS_i| <= 3 w_i |c_i|_1 max|dG| =
max|dG| / 6 for every link, and a site is a corner of at most 8 beads'
cells in these states, with |dJ| <= 1e-5 max|J| (the coupling tolerance).
One streaming step later that error sits within one site of the corners.
With FP16 storage the source pass loads, adds and stores the touched sites
again: a second rounding there.  The 1e-15 is the oracle's own: it holds
f = w_i + h in FP64, so h_orc carries the rounding of f near w_i <= 1/3.
"""
import numpy as np

import oracle
from paper_0711_2665_gb300 import inputs as inp_mod
from paper_0711_2665_gb300 import lbmd, workloads


def small_workload(**kw):
    """A small coupled case: ragged x tiles (nx = 40 is not a multiple of 32),
    a wall with a 3x3 pore, noise on, a 24-bead chain at the pore entrance."""
    base = dict(nx=40, ny=20, nz=12, n_real=1, tau=0.8, wall_x=20, pore_h=3, n_beads=24, E=0.1,
                gamma=0.1, kT=1e-4, seed=7, chain_seed=7, steps=40, precision="fp32")
    base.update(kw)
    w = workloads.get("plain_fp64_small", **base)
    return w


def make_pair(w, realization=0, inputs=None):
    inp = inputs if inputs is not None else workloads.build_inputs(w)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    o0, o1 = int(inp["offsets"][realization]), int(inp["offsets"][realization + 1])
    orc = oracle.OracleSim(workloads.oracle_params(w, realization, o1 - o0), inp["solid"])
    if o1 > o0:
        orc.set_beads(inp["r0"][o0:o1])
    return sim, orc, inp


def to_f32_state(orc):
    """The oracle's current state rounded to what the CUDA path stores."""
    f = orc.get_populations().astype(np.float32)
    r, v = orc.get_beads()
    return f, r.copy(), v.astype(np.float32).astype(np.float64)


def load_state(sim, orc, f32, r, v, step, realization=0):
    """Put the same state into a single-realization sim and into the oracle."""
    assert sim.n_real == 1
    sim.set_populations(f32[None])
    if r.shape[0]:
        sim.set_beads(r, v)
    sim.set_step(step)
    orc.set_populations(f32.astype(np.float64))
    if r.shape[0]:
        orc.set_beads(r, v)
    orc.set_step(step)


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = max(np.abs(b).max(), 1e-30)
    return float(np.abs(a - b).max() / scale)


def wave(nx, amp):
    return inp_mod.shear_wave_velocity(nx, 1, 1, amp)


def fluid_mask(inp):
    return inp["solid"] == 0


def deviations(orc, solid):
    """Oracle populations as h = f - w_i (FP64), zero at solid sites."""
    _, wts, _ = oracle.tables()
    h = orc.get_populations() - wts[:, None, None, None]
    h[:, solid != 0] = 0.0
    return h


def load_dev_state(sim, orc, h32, r, v, step, solid):
    """One state into both sides: the GPU stores the FP32 deviations h32
    exactly; the oracle gets f = w_i + h32 in FP64."""
    _, wts, _ = oracle.tables()
    assert sim.n_real == 1
    sim.set_deviations(h32[None])
    f = wts[:, None, None, None] + h32.astype(np.float64)
    f[:, solid != 0] = 0.0
    orc.set_populations(f)
    if r.shape[0]:
        sim.set_beads(r, v)
        orc.set_beads(r, v)
    sim.set_step(step)
    orc.set_step(step)


def developed_pair(w, steps=2, amp=1e-2, flow_seed=11, inputs=None):
    """Sim and oracle in the same developed state: the oracle starts from
    the equilibrium of a seeded smooth flow of amplitude amp (every site
    moves) with the workload's chain, runs `steps` steps, and its state,
    rounded to what the GPU stores (FP32 deviations and velocities), goes
    into both sides."""
    sim, orc, inp = make_pair(w, inputs=inputs)
    u = inp_mod.smooth_random_velocity(w["nx"], w["ny"], w["nz"], amp, flow_seed)
    orc.init_fluid(None, u)
    orc.step(steps)
    h32 = deviations(orc, inp["solid"]).astype(np.float32)
    r, v = orc.get_beads()
    v = v.astype(np.float32).astype(np.float64)
    load_dev_state(sim, orc, h32, r.copy(), v, steps, inp["solid"])
    return sim, orc, inp


def near_bead_sites(r, dims, pad=0):
    """Sites within 1 + pad sites of a corner of a bead's cell (periodic):
    with pad = 0 the sites the coupling reaches in one step; mask [z, y, x]."""
    nx, ny, nz = dims
    m = np.zeros((nz, ny, nx), bool)
    for p in np.asarray(r).reshape(-1, 3):
        x0 = np.floor(np.mod(p, [nx, ny, nz])).astype(int)
        xs = np.arange(x0[0] - 1 - pad, x0[0] + 3 + pad) % nx
        ys = np.arange(x0[1] - 1 - pad, x0[1] + 3 + pad) % ny
        zs = np.arange(x0[2] - 1 - pad, x0[2] + 3 + pad) % nz
        m[np.ix_(zs, ys, xs)] = True
    return m


def dev_tolerance(h_o, near=None, J_max=0.0, fp16=False):
    """Element-wise bound of one step (see the module docstring)."""
    tol = np.full(h_o.shape, 1e-5 * np.abs(h_o).max() + 1e-15)
    if fp16:
        tol += 2.0 ** -11 * np.abs(h_o) + 2.0 ** -37
    if near is not None:
        if J_max > 0.0:
            tol = tol + (8.0 / 6.0) * 1e-5 * J_max * near[None]
        if fp16:
            tol = tol + 2.0 ** -11 * np.abs(h_o) * near[None]
    return tol


def assert_dev_close(h_g, h_o, tol, fluid, label=""):
    """|h_g - h_o| <= tol at every fluid site; reports the worst ratio."""
    err = np.abs(np.asarray(h_g, np.float64) - h_o)[:, fluid]
    t = tol[:, fluid]
    ratio = float((err / t).max())
    assert ratio <= 1.0, (label, "deviations", ratio, float(err.max()), float(np.abs(h_o).max()))
    return ratio
