"""Shared helpers of the GPU tests: build a CUDA-path Simulation and an oracle
run of the same workload from the same seeded inputs, and move one state
into both."""
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
