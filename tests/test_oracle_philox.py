"""Pins of the oracle's counter-based generator and its Gaussian mapping.

* Philox4x32-10 reproduces the published known-answer vectors of Salmon,
  Moraes, Dror and Shaw (SC'11), `tests/golden/philox4x32_10_kat.json`.  A
  wrong multiplier, round-key constant, word order or hi/lo swap changes
  every output word.
* The noise mapping (the bead noise of Sec. II, Eq. 15): key =
  (seed_lo, seed_hi ^ realization), counter = (bead, step_lo, substep,
  step_hi), u_k = (top 24 bits of word k + 1/2) 2^-24, Box-Muller on (u0, u1)
  and (u2, u3).  Checked in polar form against the pinned generator's words:
  (z0, z1) has radius sqrt(-2 ln u0) and angle 2 pi u1, z2 = sqrt(-2 ln u2)
  cos(2 pi u3).  A swapped radius/angle word, a wrong bit shift or counter
  slot fails these, which the moment tests alone would not see.
"""
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")


def _kat():
    with open(GOLDEN) as fh:
        return json.load(fh)["vectors"]


@pytest.mark.parametrize("vec", _kat())
def test_philox_known_answers(orc, vec):
    ctr = [int(x, 16) for x in vec["ctr"]]
    key = [int(x, 16) for x in vec["key"]]
    out = orc.philox4x32_10(ctr, key)
    assert [f"{int(x):08x}" for x in out] == vec["out"]


def _uniform(word) -> float:
    return ((int(word) >> 8) + 0.5) / 2.0 ** 24


@pytest.mark.parametrize("seed,real,bead,step,sub", [
    (0, 0, 0, 0, 0),
    (7, 3, 11, 40, 2),
    (0x123456789ABCDEF0, 5, 999, 12345, 4),
    (3, 1, 2, (1 << 32) + 17, 1),  # a step above 2^32 reaches counter word 3
])
def test_noise_words_map_to_box_muller(orc, seed, real, bead, step, sub):
    key = [seed & 0xFFFFFFFF, (seed >> 32) ^ real]
    ctr = [bead, step & 0xFFFFFFFF, sub, step >> 32]
    x = orc.philox4x32_10(ctr, key)
    u = [_uniform(w) for w in x]
    z = orc.gauss3(seed, real, bead, step, sub)
    rad = np.sqrt(-2.0 * np.log(u[0]))
    assert np.hypot(z[0], z[1]) == pytest.approx(rad, rel=1e-12)
    ang = np.arctan2(z[1], z[0]) % (2 * np.pi)
    assert ang == pytest.approx(2 * np.pi * u[1], rel=1e-10, abs=1e-12)
    assert z[2] == pytest.approx(np.sqrt(-2.0 * np.log(u[2])) * np.cos(2 * np.pi * u[3]), rel=1e-12, abs=1e-15)


def test_uniforms_stay_inside_the_open_interval(orc):
    """The extreme words map strictly inside (0, 1), so the logarithm of
    Box-Muller stays finite: word 0 -> 2^-25, word 2^32 - 1 -> 1 - 2^-25."""
    assert _uniform(0) == 2.0 ** -25
    assert _uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -25
    z = orc.gauss3_batch(1, 0, 4096, 0, 0)
    assert np.all(np.isfinite(z))
