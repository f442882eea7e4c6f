"""Host statistics of translocation records (Sec. IV.A durations, most
probable time, scaling exponent; Sec. IV.B lambda_R), pinned by closed forms
and hand-counted cases."""
import numpy as np
import pytest

from paper_0711_2665_gb300 import transloc

REC = np.dtype([("t_origin", np.int64), ("t_first", np.int64), ("t_x", np.int64),
                ("rg_u_origin", np.float64), ("rg_t_x", np.float64), ("max_translocated", np.float64)])


def _rec(rows):
    return np.array(rows, dtype=REC)


def test_durations_and_lambda():
    rec = _rec([(0, 3, 120, 4.0, 2.8, 20), (50, 51, 90, 2.0, 1.0, 10), (0, 5, -1, 3.0, -1.0, 7)])
    tau = transloc.durations(rec)
    assert tau[0] == 120 and tau[1] == 40 and np.isnan(tau[2])
    lam = transloc.lambda_r(rec)
    assert lam[0] == pytest.approx(0.7) and lam[1] == pytest.approx(0.5) and np.isnan(lam[2])


def test_most_probable_is_the_highest_bin():
    tau = [1, 2, 2, 3, 3, 3, 4, 10]
    edges = np.arange(0.5, 11.0, 1.0)
    assert transloc.most_probable(tau, edges) == 3.0
    counts, e = transloc.histogram(tau, edges)
    assert counts.sum() == len(tau) and counts.max() == 3
    # ties go to the first bin; an empty or a constant sample
    assert transloc.most_probable([1, 1, 5, 5], np.array([0.5, 1.5, 2.5, 3.5, 4.5, 5.5])) == 1.0
    assert np.isnan(transloc.most_probable([np.nan]))
    assert transloc.most_probable([7, 7, 7]) == 7.0


def test_most_probable_of_a_skewed_law():
    """Gamma(k=6, theta=50) has its mode at (k-1) theta = 250 below its mean
    k theta = 300: the estimate lands near the mode, not the mean.  The
    density is flat at the mode, so one sample's highest bin scatters by
    some 20 about it; the mean over eight samples scatters far less."""
    mps = []
    for seed in range(8):
        tau = np.random.default_rng(seed).gamma(6.0, 50.0, size=200000)
        mps.append(transloc.most_probable(tau))
    mps = np.array(mps)
    assert np.abs(mps - 250.0).max() < 40.0
    assert abs(mps.mean() - 250.0) < 12.0


def test_exponent_of_an_exact_power_law():
    n = np.array([20, 40, 60, 80, 100, 140, 200])
    fit = transloc.scaling_exponent(n, 3.0 * n ** 1.28)
    assert fit["alpha"] == pytest.approx(1.28, abs=1e-12)
    assert fit["prefactor"] == pytest.approx(3.0, rel=1e-10)
    assert fit["alpha_stderr"] < 1e-10
    two = transloc.scaling_exponent([10, 1000], [5.0, 5.0 * 100 ** 1.5])
    assert two["alpha"] == pytest.approx(1.5) and np.isnan(two["alpha_stderr"])
    with pytest.raises(ValueError):
        transloc.scaling_exponent([10], [5.0])


def test_exponent_with_scatter_and_its_error():
    """log-normal scatter of 5%: the fit stays within four standard errors of
    the true exponent, and the error matches the textbook formula."""
    rng = np.random.default_rng(3)
    n = np.repeat([20, 40, 80, 160, 320], 4).astype(float)
    tau = 2.0 * n ** 1.36 * np.exp(0.05 * rng.standard_normal(n.size))
    fit = transloc.scaling_exponent(n, tau)
    assert abs(fit["alpha"] - 1.36) < 4 * fit["alpha_stderr"]
    x, y = np.log(n), np.log(tau)
    slope, icpt = np.polyfit(x, y, 1)
    res = y - (icpt + slope * x)
    se = np.sqrt(res @ res / (n.size - 2) / ((x - x.mean()) ** 2).sum())
    assert fit["alpha"] == pytest.approx(slope, rel=1e-10)
    assert fit["alpha_stderr"] == pytest.approx(se, rel=1e-8)


def test_summary_groups_by_length():
    counts = np.array([20, 20, 20, 40, 40, 40])
    rec = _rec([(0, 1, 100, 2.0, 1.5, 20), (0, 1, 110, 2.0, 1.5, 20), (0, 1, 100, 2.0, 1.5, 20),
                (0, 1, 250, 3.0, 2.0, 40), (0, 1, 250, 3.0, 2.0, 40), (0, 1, -1, 3.0, -1.0, 31)])
    s = transloc.summarize(counts, rec, bins=np.arange(0.0, 400.0, 20.0))
    a, b = s["by_length"][20], s["by_length"][40]
    assert a["events"] == 3 and a["completed"] == 3 and b["completed"] == 2
    assert a["tau_mean"] == pytest.approx(310 / 3) and a["tau_most_probable"] == 110.0
    assert b["tau_most_probable"] == 250.0
    assert a["lambda_r_mean"] == pytest.approx(0.75) and b["lambda_r_mean"] == pytest.approx(2 / 3)
    assert s["fit"]["alpha"] == pytest.approx(np.log(250 / 110) / np.log(2))
