"""The other forms of the lattice pass against the scalar one (one site per
thread, tiles by > 0): the kernel fed by tensor copies (by = 0) and the one
with two x sites per thread (by < 0).  The per-site arithmetic is the same,
so every state they produce is the same bit for bit, here over coupled steps
with the chain, in FP32 and FP16 storage: rows of 40 sites (six rows per copy
group, the last group ragged; 20 of a warp's 32 pairs), 42 sites (a pair
tile straddling the wall plane at x = 21), the 64-realization ensemble, the
full 4.19M-site lattice and a slab."""
import numpy as np
import pytest

from gpu_helpers import small_workload
from paper_0711_2665_gb300 import dist as pdist
from paper_0711_2665_gb300 import inputs as inp_mod
from paper_0711_2665_gb300 import lbmd, workloads

pytestmark = pytest.mark.gpu


def _pair(w, steps, tiles_a, tiles_b, flow=True):
    inp = workloads.build_inputs(w)
    out = []
    for tiles in (tiles_a, tiles_b):
        sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
        sim.set_tiles(*tiles)
        if flow:
            u = np.stack([inp_mod.smooth_random_velocity(w["nx"], w["ny"], w["nz"], 1e-2, 7 + r)
                          for r in range(w["n_real"])])
            sim.init_fluid(None, u)
        sim.step(steps)
        sim.check()
        out.append((sim.get_deviations(), *sim.get_beads(), sim.diagnostics(steps)))
        sim.close()
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp16dev"])
@pytest.mark.parametrize("groups", [1, 3, 16])
def test_tensor_copy_pass_is_bit_identical_small(precision, groups):
    w = small_workload(precision=precision)
    (ha, ra, va, da), (hb, rb, vb, db) = _pair(w, 12, (4, 4), (0, groups))
    assert np.array_equal(ha, hb)
    assert np.array_equal(ra, rb) and np.array_equal(va, vb)
    # The fluid sums differ only in how sites are grouped into FP32 partials
    # before the exact fixed-point total: a thread adds k <= groups + 4 sites
    # per kernel, so each side is within k 2^-24 sum|drho| of the exact sum,
    # with sum|drho| <= sum over sites and links of |f_i - w_i| (taken from
    # the last state, four times over for the larger early transients).
    _sums_close(da, db, ha, groups + 4)


def test_tensor_copy_pass_ensemble_and_full_lattice():
    w = workloads.get("ensemble_fp32")
    (ha, ra, va, _), (hb, rb, vb, _) = _pair(w, 4, (4, 2), (0, 8), flow=False)
    assert np.array_equal(ha, hb) and np.array_equal(ra, rb) and np.array_equal(va, vb)
    w = workloads.get("lattice_4m_fp32")
    (ha, ra, va, _), (hb, rb, vb, _) = _pair(w, 3, (4, 4), (0, 16), flow=False)
    assert np.array_equal(ha, hb) and np.array_equal(ra, rb) and np.array_equal(va, vb)


def test_tensor_copy_pass_in_a_slab():
    """Two slabs of 61 planes of a 122-plane lattice: each slab's 64 local
    planes (256-byte rows) fit the tensor-copy kernel, the whole lattice's
    488-byte rows do not; the split equals the whole lattice bit for bit."""
    w = small_workload(nx=122, ny=16, nz=12, wall_x=60)
    inp = workloads.build_inputs(w)
    whole = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    sims = []
    for rank in range(2):
        s = lbmd.Simulation(pdist.slab_workload(w, rank, 2), inp["solid"], inp["offsets"], inp["r0"])
        s.set_tiles(0, 4)
        sims.append(s)
    for _ in range(6):
        whole.step(1)
        pdist.slab_step_local(sims)
    h = whole.get_deviations()[0]
    for s, (x0, wd) in zip(sims, pdist.slab_partition(w["nx"], 2)):
        same = bool(np.array_equal(s.get_deviations()[0][:, :, :, 1:wd + 1], h[:, :, :, x0:x0 + wd]))
        assert same, (x0, wd)


def _sums_close(da, db, ha, k):
    """Fluid sums grouped differently into FP32 partials (k sites a thread at
    most): each within k 2^-24 sum|drho| of the exact sum."""
    tol = 2 * k * 2.0 ** -24 * 4.0 * float(np.abs(ha.astype(np.float64)).sum())
    assert np.abs(da["mass"] - db["mass"]).max() <= tol
    assert np.abs(da["p_fluid"] - db["p_fluid"]).max() <= tol


@pytest.mark.parametrize("precision", ["fp32", "fp16dev"])
@pytest.mark.parametrize("tiles", [(-1, 1), (-4, 3), (-8, 16)])
@pytest.mark.parametrize("nx", [40, 42])
def test_paired_pass_is_bit_identical_small(precision, tiles, nx):
    w = small_workload(precision=precision, nx=nx, wall_x=nx // 2)
    (ha, ra, va, da), (hb, rb, vb, db) = _pair(w, 12, (4, 4), tiles)
    assert np.array_equal(ha, hb)
    assert np.array_equal(ra, rb) and np.array_equal(va, vb)
    _sums_close(da, db, ha, 2 * tiles[1] + 4)


def test_paired_pass_ensemble_full_lattice_and_slab():
    w = workloads.get("ensemble_fp32")
    (ha, ra, va, _), (hb, rb, vb, _) = _pair(w, 4, (4, 2), (-4, 4), flow=False)
    assert np.array_equal(ha, hb) and np.array_equal(ra, rb) and np.array_equal(va, vb)
    for prec in ("fp32", "fp16dev"):
        w = workloads.get("lattice_4m_fp32", precision=prec)
        (ha, ra, va, _), (hb, rb, vb, _) = _pair(w, 3, (4, 4), (-2, 8), flow=False)
        assert np.array_equal(ha, hb) and np.array_equal(ra, rb) and np.array_equal(va, vb), prec
    # two slabs of a 122-plane lattice: 64 local planes each (even)
    w = small_workload(nx=122, ny=16, nz=12, wall_x=60)
    inp = workloads.build_inputs(w)
    whole = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    sims = []
    for rank in range(2):
        s = lbmd.Simulation(pdist.slab_workload(w, rank, 2), inp["solid"], inp["offsets"], inp["r0"])
        s.set_tiles(-4, 2)
        sims.append(s)
    for _ in range(6):
        whole.step(1)
        pdist.slab_step_local(sims)
    h = whole.get_deviations()[0]
    for s, (x0, wd) in zip(sims, pdist.slab_partition(w["nx"], 2)):
        same = bool(np.array_equal(s.get_deviations()[0][:, :, :, 1:wd + 1], h[:, :, :, x0:x0 + wd]))
        assert same, (x0, wd)


def test_paired_pass_needs_an_even_row():
    """An odd nx has no aligned pairs; blocks hold at most 256 threads (three
    per SM at 80 registers), so by = -16 is refused too."""
    w = small_workload(nx=41, wall_x=20)
    inp = workloads.build_inputs(w)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    with pytest.raises(lbmd.LbmdError):
        sim.set_tiles(-4, 4)
    w = small_workload()
    inp = workloads.build_inputs(w)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    sim.set_tiles(-8, 4)
    with pytest.raises(lbmd.LbmdError):
        sim.set_tiles(-16, 4)


def test_tensor_copy_pass_needs_a_fitting_lattice():
    w = small_workload(nx=42, wall_x=21)  # 168-byte FP32 rows: not a multiple of 16 bytes
    inp = workloads.build_inputs(w)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    with pytest.raises(lbmd.LbmdError):
        sim.set_tiles(0, 4)
