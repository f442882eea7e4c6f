"""The six named workloads of the coupled LB-MD step, and how to build them.

Each workload is a plain dict of parameters (lattice units) plus a recipe for
its seeded inputs; it carries no arithmetic of the method.  Parameters the
workload statements leave open are filled with the readings listed in the
design notes: tau = 0.8 (kinematic viscosity 0.1, Sec. IV) where no tau is
given; bending constant kappa = 1e-3, ten times the paper's kT = 1e-4, which
gives the persistence length of about 10 monomers stated in Sec. IV; bead-wall
WCA with the bead-bead sigma and eps; M = 5 and M^b = 20 (Sec. II).

  plain_fp64_small   32x16x16, tau 1, wall x=16, 3x3 pore, N=20, E=0.05,
                     gamma 0.1, noise off, 1000 steps
  plain_fp32         128x64x64, tau 0.8, wall x=64, 5x5 pore, N=400 SAW,
                     E=0.1, gamma 0.1, kT=1e-4, 10000 steps
  ensemble_fp32      64 realizations of 64x32x32, wall x=32, 3x3 pore,
                     N ~ U{20..200}, E=0.05, gamma 0.1, kT=1e-4, 5000 steps
  fp16dev            256x128x128, wall x=128, 3x3 pore, N=1000, E=0.1,
                     gamma 0.2, kT=1e-4, populations as FP16 deviations
  lattice_4m_fp32    the same 256x128x128 lattice (4.19M sites) and chain
                     with FP32 storage: the plain step on the largest
                     single-lattice configuration
  adjoint            96x48x48, wall x=48, 4x4 pore, N=100, E=0.1,
                     gamma 0.1, kT=1e-4, K=200, checkpoints every 20
"""
from __future__ import annotations

import numpy as np

from . import inputs

COMMON = dict(k_bond=100.0, r0=1.0, kappa_bend=1e-3, lj_sigma=1.0, lj_eps=1.0,
              wall_sigma=1.0, wall_eps=1.0, md_outer=5, md_inner=20,
              body_force=(0.0, 0.0, 0.0))

WORKLOADS = {
    "plain_fp64_small": dict(COMMON, nx=32, ny=16, nz=16, n_real=1, tau=1.0, wall_x=16, pore_h=3,
                             n_beads=20, E=0.05, gamma=0.1, kT=0.0, seed=0, chain_seed=0,
                             steps=1000, precision="fp32"),
    "plain_fp32": dict(COMMON, nx=128, ny=64, nz=64, n_real=1, tau=0.8, wall_x=64, pore_h=5,
                       n_beads=400, E=0.1, gamma=0.1, kT=1e-4, seed=1, chain_seed=1,
                       steps=10000, precision="fp32"),
    "ensemble_fp32": dict(COMMON, nx=64, ny=32, nz=32, n_real=64, tau=0.8, wall_x=32, pore_h=3,
                          n_beads=(20, 200), E=0.05, gamma=0.1, kT=1e-4, seed=2, chain_seed=2,
                          steps=5000, precision="fp32"),
    "fp16dev": dict(COMMON, nx=256, ny=128, nz=128, n_real=1, tau=0.8, wall_x=128, pore_h=3,
                    n_beads=1000, E=0.1, gamma=0.2, kT=1e-4, seed=3, chain_seed=3,
                    steps=20000, precision="fp16dev"),
    "lattice_4m_fp32": dict(COMMON, nx=256, ny=128, nz=128, n_real=1, tau=0.8, wall_x=128, pore_h=3,
                            n_beads=1000, E=0.1, gamma=0.2, kT=1e-4, seed=3, chain_seed=3,
                            steps=20000, precision="fp32"),
    "adjoint": dict(COMMON, nx=96, ny=48, nz=48, n_real=1, tau=0.8, wall_x=48, pore_h=4,
                    n_beads=100, E=0.1, gamma=0.1, kT=1e-4, seed=4, chain_seed=4,
                    steps=200, checkpoint_every=20, precision="fp32"),
}


def get(name: str, **overrides) -> dict:
    w = dict(WORKLOADS[name])
    w.update(overrides)
    w["name"] = name
    return w


def bead_counts(w: dict) -> np.ndarray:
    """Beads per realization (explicit "bead_counts", a (lo, hi) range drawn
    per realization, or one count for all)."""
    if w.get("bead_counts") is not None:
        return np.asarray(w["bead_counts"], dtype=np.int32)
    nb = w["n_beads"]
    if isinstance(nb, (tuple, list)):
        return inputs.chain_lengths(w["n_real"], nb[0], nb[1], w["chain_seed"])
    return np.full(w["n_real"], int(nb), dtype=np.int32)


def build_inputs(w: dict) -> dict:
    """Solid mask, bead counts / CSR offsets and initial chains of a workload."""
    nx, ny, nz = w["nx"], w["ny"], w["nz"]
    solid = w.get("solid")
    if solid is None:
        solid = inputs.pore_wall_mask(nx, ny, nz, w["wall_x"], w["pore_h"])
    counts = bead_counts(w)
    offsets = np.zeros(len(counts) + 1, dtype=np.int32)
    offsets[1:] = np.cumsum(counts)
    chains = []
    for r, n in enumerate(counts):
        seed = int(w["chain_seed"]) * 100003 + r
        chains.append(inputs.chain_walk(int(n), (nx, ny, nz), w["wall_x"], solid, seed,
                                        bond=w["r0"]))
    r0 = np.concatenate(chains, axis=0) if chains else np.zeros((0, 3))
    return dict(solid=solid, counts=counts, offsets=offsets, r0=r0)


def oracle_params(w: dict, realization: int = 0, n_beads: int | None = None) -> dict:
    """Parameter dict in the oracle's vocabulary for one realization."""
    keys = ("nx", "ny", "nz", "tau", "body_force", "wall_x", "pore_h", "k_bond", "r0",
            "kappa_bend", "lj_sigma", "lj_eps", "wall_sigma", "wall_eps", "E", "gamma", "kT",
            "md_outer", "md_inner", "seed")
    p = {k: w[k] for k in keys}
    p["realization"] = int(w.get("real_base", 0)) + realization
    for k, d in (("interp", 0), ("integrator", 0), ("lb_kT", 0.0)):
        p[k] = w.get(k, d)
    p["n_beads"] = int(n_beads if n_beads is not None else bead_counts(w)[realization])
    return p
