"""An ensemble split into blocks of realizations (real_base = first global
index, inputs sliced from the unsplit ones) evolves exactly as the unsplit
ensemble: the per-realization state after several coupled steps is
bit-identical.  This is what lets ranks of a multi-GPU job shard an
ensemble without any collective on the data path."""
import numpy as np
import pytest

from paper_0711_2665_gb300 import dist as pdist
from paper_0711_2665_gb300 import lbmd, workloads

pytestmark = pytest.mark.gpu


def test_split_ensemble_matches_unsplit():
    w = workloads.get("ensemble_fp32", nx=40, ny=20, nz=12, wall_x=20, n_real=5, n_beads=(6, 14))
    full_inp = workloads.build_inputs(w)
    whole = lbmd.Simulation(w, full_inp["solid"], full_inp["offsets"], full_inp["r0"])
    whole.set_md_shape(4, 1)
    whole.step(6)
    dev = whole.get_deviations()
    r_all, v_all = whole.get_beads()
    for rank in range(2):
        wr = pdist.rank_workload(w, rank, 2)
        inp = pdist.rank_inputs(wr, workloads.build_inputs)
        part = lbmd.Simulation(wr, inp["solid"], inp["offsets"], inp["r0"])
        part.set_md_shape(4, 1)
        part.step(6)
        lo, hi = wr["shard"]
        b0, b1 = int(full_inp["offsets"][lo]), int(full_inp["offsets"][hi])
        assert np.array_equal(part.get_deviations(), dev[lo:hi])
        r, v = part.get_beads()
        assert np.array_equal(r, r_all[b0:b1]) and np.array_equal(v, v_all[b0:b1])


def test_packed_chains_match_chains_alone():
    """Chains of very different lengths on clusters of 4 blocks of Nc = 10
    beads: a chain takes ceil(N / 10) blocks, so the 25- and the 6-bead chain
    share a cluster.  Each realization evolves exactly as it does alone (a
    one-realization shard with the same noise stream)."""
    counts = [40, 6, 25, 12, 33]
    w = workloads.get("ensemble_fp32", nx=40, ny=20, nz=12, wall_x=20, n_real=len(counts), bead_counts=counts)
    full_inp = workloads.build_inputs(w)
    whole = lbmd.Simulation(w, full_inp["solid"], full_inp["offsets"], full_inp["r0"])
    whole.set_md_shape(4, 4)
    whole.step(8)
    whole.check()
    dev = whole.get_deviations()
    r_all, v_all = whole.get_beads()
    for r in range(len(counts)):
        wr = pdist.rank_workload(w, r, len(counts))
        inp = pdist.rank_inputs(wr, workloads.build_inputs)
        alone = lbmd.Simulation(wr, inp["solid"], inp["offsets"], inp["r0"])
        alone.set_md_shape(4, 4)
        alone.step(8)
        b0, b1 = int(full_inp["offsets"][r]), int(full_inp["offsets"][r + 1])
        assert np.array_equal(alone.get_deviations(), dev[r:r + 1]), r
        ra, va = alone.get_beads()
        assert np.array_equal(ra, r_all[b0:b1]) and np.array_equal(va, v_all[b0:b1]), r
        alone.close()
