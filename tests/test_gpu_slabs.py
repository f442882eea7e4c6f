"""One lattice split into x-slabs (the paper's domain decomposition, Sec. III,
along x), each slab its own handle, against the unsplit lattice: after K
coupled steps every slab's own planes and the replicated chain equal the
whole lattice's bit for bit.  The slabs live in one process on one device,
and the exchange is a copy between their buffers (dist.slab_step_local); the
transport over ranks is tested on CPU ranks in test_dist_slabs_gloo.py."""
import numpy as np
import pytest

from gpu_helpers import small_workload
from paper_0711_2665_gb300 import dist as pdist
from paper_0711_2665_gb300 import inputs as inp_mod
from paper_0711_2665_gb300 import lbmd, workloads

pytestmark = pytest.mark.gpu


def _run(w, world, steps, flow=True, shape=(2, 2)):
    inp = workloads.build_inputs(w)
    u = inp_mod.smooth_random_velocity(w["nx"], w["ny"], w["nz"], 1e-2, 3) if flow else None
    whole = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    whole.set_md_shape(*shape)
    if flow:
        whole.init_fluid(None, u[None])
    parts = pdist.slab_partition(w["nx"], world)
    sims = []
    for rank in range(world):
        ws = pdist.slab_workload(w, rank, world)
        s = lbmd.Simulation(ws, inp["solid"], inp["offsets"], inp["r0"])
        s.set_md_shape(*shape)
        if flow:  # the slab's planes and ghosts of the same flow
            x0, wd = parts[rank]
            xs = np.arange(x0 - 1, x0 + wd + 2) % w["nx"]
            s.init_fluid(None, u[:, :, :, xs][None])
        sims.append(s)
    for _ in range(steps):
        whole.step(1)
        pdist.slab_step_local(sims)
    return whole, sims, parts


def _assert_same(whole, sims, parts):
    h = whole.get_deviations()[0]
    for s, (x0, wd) in zip(sims, parts):
        hs = s.get_deviations()[0]
        same = bool(np.array_equal(hs[:, :, :, 1:wd + 1], h[:, :, :, x0:x0 + wd]))
        diff = float(np.abs(hs[:, :, :, 1:wd + 1] - h[:, :, :, x0:x0 + wd]).max())
        assert same, ("slab populations differ", x0, wd, diff)
    rw, vw = whole.get_beads()
    for s in sims:
        r, v = s.get_beads()
        same = bool(np.array_equal(r, rw) and np.array_equal(v, vw))
        assert same, ("beads differ", float(np.abs(r - rw).max()), float(np.abs(v - vw).max()))
        s.check()
    # fluid sums add up over the slabs; bead sums are every slab's
    dw = whole.diagnostics()[0]
    ds = [s.diagnostics()[0] for s in sims]
    assert np.allclose(sum(d["mass"] for d in ds), dw["mass"], rtol=1e-12)
    assert np.allclose(sum(d["p_fluid"] for d in ds), dw["p_fluid"], rtol=1e-6, atol=1e-9)
    for d in ds:
        same = bool(np.array_equal(d["p_beads"], dw["p_beads"]) and np.array_equal(d["com"], dw["com"]))
        assert same, "bead sums differ"


@pytest.mark.parametrize("world", [1, 2, 3])
def test_slabs_match_the_whole_lattice(world):
    """40x20x12 with the wall at x = 20 and the chain at the pore entrance,
    under a seeded flow: the chain's cells straddle the slab boundary at
    x = 20 (two slabs) or lie in the middle slab (three slabs of 14, 13, 13
    planes); one slab is the whole lattice exchanging with itself."""
    w = small_workload()
    whole, sims, parts = _run(w, world, steps=12)
    _assert_same(whole, sims, parts)


def test_slabs_fp16_storage():
    w = small_workload(precision="fp16dev")
    whole, sims, parts = _run(w, 2, steps=8)
    _assert_same(whole, sims, parts)


def test_slabs_full_size_lattice():
    """The 256x128x128 lattice with the 1000-bead chain in two slabs."""
    w = workloads.get("lattice_4m_fp32")
    whole, sims, parts = _run(w, 2, steps=3, flow=False, shape=(2, 16))
    _assert_same(whole, sims, parts)


def test_slab_calls_are_checked():
    w = small_workload()
    inp = workloads.build_inputs(w)
    whole = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    with pytest.raises(lbmd.LbmdError):
        whole.slab_gather()
    s = lbmd.Simulation(pdist.slab_workload(w, 0, 2), inp["solid"], inp["offsets"], inp["r0"])
    for call in (lambda: s.step(1), lambda: s.step_loop(2), lambda: s.observables(), lambda: s.set_graph(2)):
        with pytest.raises(lbmd.LbmdError):
            call()
    with pytest.raises(lbmd.LbmdError):  # a slab of one plane
        lbmd.Simulation(dict(w, slab=(0, 1)), inp["solid"], inp["offsets"], inp["r0"])
