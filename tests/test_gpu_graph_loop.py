"""The device-side step loop (lbmd_step_loop: one CUDA-graph launch whose
conditional WHILE node repeats two coupled steps) gives the same state, bit for
bit, as steps launched one by one and as the unrolled step graph, for even and
odd step counts, on an ensemble with uneven chains."""
import numpy as np
import pytest

from paper_0711_2665_gb300 import lbmd, workloads

pytestmark = pytest.mark.gpu


def _ens():
    w = workloads.get("ensemble_fp32", nx=40, ny=20, nz=12, wall_x=20, n_real=3, n_beads=(6, 14))
    inp = workloads.build_inputs(w)
    return w, inp


def _state(sim):
    r, v = sim.get_beads()
    return sim.get_deviations(), r, v, sim.step_count


def _same(a, b):
    assert a[3] == b[3]
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("n", [1, 2, 7, 12])
def test_loop_matches_eager_and_unrolled_graph(n):
    w, inp = _ens()
    eager = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    eager.step(n)
    loop = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    loop.step_loop(n)
    unrolled = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    unrolled.set_graph(2)
    unrolled.step(n)
    s = _state(eager)
    _same(s, _state(loop))
    _same(s, _state(unrolled))


def test_loop_relaunch_and_realign():
    w, inp = _ens()
    eager = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    loop = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    for n in (4, 3, 6, 0, 5):  # odd counts leave the buffers swapped; the next call realigns
        eager.step(n)
        loop.step_loop(n)
    _same(_state(eager), _state(loop))
    loop.set_tiles(4, 4)  # drops the loop graph; it is captured again
    eager.set_tiles(4, 4)
    eager.step(4)
    loop.step_loop(4)
    _same(_state(eager), _state(loop))
    loop.check()
