"""The device generator of the noise against the oracle's, through the C ABI.

* Raw Philox4x32-10 words: bit for bit, on the published known-answer vectors
  and on 2^16 random (counter, key) pairs.  The oracle's generator is pinned
  to the known answers on the CPU (tests/test_oracle_philox.py), so a shared
  misreading of the generator would fail here or there.
* Bead-noise normals (Sec. II, Eq. 15): the device maps the words in FP32.
  Tolerance, from that arithmetic: u = (top 24 bits + 1/2) 2^-24 rounds to
  FP32 with an error of at most 2^-25 (the half is lost once the top bits
  reach 2^23), which moves the Box-Muller radius sqrt(-2 ln u) by at most
  sqrt(2 * 2^-25) = 2^-12 (at u -> 1, where the radius is itself near 0), and
  the angle 2 pi u by 2 pi 2^-25; logf, sqrtf and sincospif add a few ulps.
  So |z_gpu - z_orc| <= 2^-12 + 4e-6 max(1, |z|), and the median error stays
  at FP32 rounding (1e-6).
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")


def test_device_philox_matches_known_answers_and_oracle(orc):
    from paper_0711_2665_gb300 import lbmd
    with open(GOLDEN) as fh:
        kat = json.load(fh)["vectors"]
    rows = [[int(x, 16) for x in v["ctr"]] + [int(x, 16) for x in v["key"]] for v in kat]
    got = lbmd.philox4x32_10(np.array(rows, dtype=np.uint32))
    for g, v in zip(got, kat):
        assert [f"{int(x):08x}" for x in g] == v["out"]
    rng = np.random.default_rng(2024)
    ck = rng.integers(0, 2 ** 32, size=(1 << 16, 6), dtype=np.uint64).astype(np.uint32)
    got = lbmd.philox4x32_10(ck)
    want = np.array([orc.philox4x32_10(r[:4], r[4:]) for r in ck[:4096]])
    assert np.array_equal(got[:4096], want)
    # the rest against a second oracle pass over a strided sample
    idx = np.arange(4096, 1 << 16, 61)
    want = np.array([orc.philox4x32_10(ck[i, :4], ck[i, 4:]) for i in idx])
    assert np.array_equal(got[idx], want)


@pytest.mark.parametrize("seed,real,step,sub", [(7, 3, 40, 2), (0x123456789ABCDEF0, 5, (1 << 32) + 17, 4),
                                                (1, 0, 0, 0)])
def test_device_bead_noise_matches_oracle(orc, seed, real, step, sub):
    from paper_0711_2665_gb300 import lbmd
    n = 20000
    zg = lbmd.noise_gauss3(seed, real, 0, n, step, sub).astype(np.float64)
    zo = orc.gauss3_batch(seed, real, n, step, sub)
    err = np.abs(zg - zo)
    tol = 2.0 ** -12 + 4e-6 * np.maximum(1.0, np.abs(zo))
    assert np.all(err <= tol), float((err - tol).max())
    assert np.median(err) <= 1e-6
    # an offset first bead draws the same numbers as the full batch
    zg2 = lbmd.noise_gauss3(seed, real, 100, 50, step, sub)
    assert np.array_equal(zg2, zg[100:150].astype(np.float32))
