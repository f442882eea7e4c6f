"""The state transfer through the C ABI rounds exactly as its FP64 definition.

The library holds the deviations h = f - w_i (Sec. II: f_i near the weights
w_i of the D3Q19 equilibrium at rest).  lbmd_set_populations stores
h = float(double(f) - w_i) and lbmd_get_populations returns
f = float(double(h) + w_i), w_i the double nearest the weight.  The kernels
evaluate both in FP32 with error-free sums and fall back to FP64 only near a
rounding midpoint; these tests check every element bit for bit against
numpy's FP64 evaluation, on deviations of every scale from 1e-38 to 0.2,
zeros, and populations equal to float(w_i) and its neighbours.  With FP16
storage the stored value is h 2^12 rounded to FP16 (round to nearest even),
which numpy's float16 conversion gives independently."""
import numpy as np
import pytest

from gpu_helpers import small_workload
from paper_0711_2665_gb300 import lbmd, workloads

pytestmark = pytest.mark.gpu

WD = np.array([1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12)[:, None, None, None]


def _bits_equal(a, b, mask):
    a = np.ascontiguousarray(a[:, mask], dtype=np.float32).view(np.uint32)
    b = np.ascontiguousarray(b[:, mask], dtype=np.float32).view(np.uint32)
    bad = np.flatnonzero(a != b)
    return bad.size, (a.ravel()[bad[:5]].view(np.float32).tolist(), b.ravel()[bad[:5]].view(np.float32).tolist())


def _fp16_stored(h32):
    """What FP16 deviation storage holds for h: (h 2^12) rounded to FP16, scaled back."""
    return ((h32 * np.float32(4096.0)).astype(np.float16).astype(np.float32) / np.float32(4096.0)).astype(np.float32)


@pytest.mark.parametrize("precision", ["fp32", "fp16dev"])
def test_state_conversions_round_as_their_fp64_definition(precision):
    w = small_workload(precision=precision)
    inp = workloads.build_inputs(w)
    sim = lbmd.Simulation(w, inp["solid"], inp["offsets"], inp["r0"])
    fluid = inp["solid"] == 0
    shape = sim.get_deviations()[0].shape
    rng = np.random.default_rng(11)

    # deviations -> populations: f = float(double(h) + w_i)
    h = rng.choice([-1.0, 1.0], size=shape) * 10.0 ** rng.uniform(-38.0, -0.7, size=shape)
    h.reshape(-1)[::97] = 0.0
    h[:, ::3, ::2, ::5] = (WD.astype(np.float32).astype(np.float64) - WD)[:, :, :, :]  # f = float(w_i) exactly
    h32 = h.astype(np.float32)
    sim.set_deviations(h32[None])
    h_held = sim.get_deviations()[0]
    if precision == "fp16dev":
        n, ex = _bits_equal(h_held, _fp16_stored(h32), fluid)
        assert n == 0, ("stored deviations", n, ex)
    f_want = (h_held.astype(np.float64) + WD).astype(np.float32)
    n, ex = _bits_equal(sim.get_populations()[0], f_want, fluid)
    assert n == 0, ("populations", n, ex)

    # populations -> deviations: h = float(double(f) - w_i)
    f = WD * (1.0 + rng.choice([-1.0, 1.0], size=shape) * 10.0 ** rng.uniform(-12.0, -0.7, size=shape))
    f32 = f.astype(np.float32)
    a = WD.astype(np.float32) * np.ones(shape, dtype=np.float32)
    f32[:, ::4, ::3, ::2] = a[:, ::4, ::3, ::2]
    f32[:, 1::4, ::3, ::2] = np.nextafter(a, np.float32(1.0))[:, 1::4, ::3, ::2]
    f32[:, 2::4, ::3, ::2] = np.nextafter(a, np.float32(0.0))[:, 2::4, ::3, ::2]
    sim.set_populations(f32[None])
    h_want = (f32.astype(np.float64) - WD).astype(np.float32)
    if precision == "fp16dev":
        h_want = _fp16_stored(h_want)
    n, ex = _bits_equal(sim.get_deviations()[0], h_want, fluid)
    assert n == 0, ("deviations", n, ex)
    sim.close()
