"""Pins of the law fitter (§2 Eq. 2, §5 Table tab:fit, §6 branch band)."""
import json
import math
import os

import numpy as np
import pytest

from paper_2606_22423_gb300 import lawfit

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "tab_fit.json")))


def test_table_rows_imply_each_machines_read_bandwidth():
    # b* = 8 beta / T_dec, so every row of one machine implies the same beta
    betas = {}
    for row in GOLD["rows"]:
        betas.setdefault(row["machine"], []).append(
            lawfit.implied_beta(row["t_dec_gvals"] * 1e9, row["b_star"]) / 1e9)
    x86, m4 = np.array(betas["x86"]), np.array(betas["M4"])
    lo, hi = GOLD["beta_scan_gbs"]["x86"]
    # the three x86 rows agree to ~1% and sit at the low end of the stated range
    assert np.ptp(x86) / x86.mean() < 0.02 and lo - 0.5 <= x86.mean() <= hi
    # M4 rows reproduce beta_scan ~ 70 GB/s, not the 93 GB/s Triad figure
    assert np.ptp(m4) / m4.mean() < 0.02 and abs(m4.mean() - GOLD["beta_scan_gbs"]["M4"]) < 1.5
    # ridge formula round-trips
    for row in GOLD["rows"]:
        beta = lawfit.implied_beta(row["t_dec_gvals"] * 1e9, row["b_star"])
        assert lawfit.ridge(row["t_dec_gvals"] * 1e9, beta) == pytest.approx(row["b_star"])


def test_fastlanes_limit_saturates_at_three_bits():
    fl = GOLD["fastlanes_limit"]
    t, beta = fl["t_dec_gvals"] * 1e9, fl["beta_gbs"] * 1e9
    assert lawfit.law_f(t, fl["saturates_at_b"], beta) == 1.0
    assert lawfit.law_f(t, 2, beta) < 1.0
    # the ridge the formula gives (the text's "about 1 bit" does not follow from it)
    assert lawfit.ridge(t, beta) == pytest.approx(8 * 52 / 140)


def test_law_shape():
    beta, t = 7e12, 3e12
    b = np.arange(1, 33)
    f = lawfit.law_f(t, b, beta)
    bstar = lawfit.ridge(t, beta)
    assert np.all(np.diff(f) >= 0) and f[-1] == 1.0
    np.testing.assert_allclose(f[b < bstar], t * b[b < bstar] / (8 * beta))
    assert np.all(f[b >= bstar] == 1.0)


@pytest.mark.parametrize("t_true", [5e11, 2.5e12, 9e12])
def test_fit_recovers_the_parameter_of_noise_free_points(t_true):
    beta = 7.3e12
    b = np.arange(1, 33)
    f = lawfit.law_f(t_true, b, beta)
    t, err = lawfit.fit_tdec(b, f, beta)
    assert t == pytest.approx(t_true, rel=1e-3) and err < 1e-4
    t2, rms = lawfit.fit_tdec_lsq(b, f, beta)
    assert t2 == pytest.approx(t_true, rel=2e-3)


def test_fit_median_is_robust_to_outliers():
    beta, t_true = 7e12, 2e12
    b = np.arange(1, 33)
    f = lawfit.law_f(t_true, b, beta)
    f[[0, 5, 9]] = [0.9, 0.01, 0.99]        # three wild points
    t, _ = lawfit.fit_tdec(b, f, beta)
    assert t == pytest.approx(t_true, rel=0.02)


def test_branch_band_edges_match_the_printed_model_pairs():
    for machine in ("x86", "M4"):
        lo, hi = GOLD["branch_band_model"][machine]
        assert lo + hi == pytest.approx(1.0)          # the printed pairs are symmetric
        k = lo * (1 - lo)
        e = lawfit.band_edges(k)
        assert e[0] == pytest.approx(lo) and e[1] == pytest.approx(hi)
    assert lawfit.band_edges(0.3) is None


def test_branch_model_fit_recovers_parabola_and_divergence():
    s = np.array([1e-3, 1e-2, 0.1, 0.3, 0.5, 0.7, 0.9, 0.99, 1.0])
    tb = 2.0 + 8.0 * s * (1 - s)
    fit = lawfit.fit_branch_models(s, tb, np.full_like(s, 3.0))
    assert fit["parabola"]["A"] == pytest.approx(2.0) and fit["parabola"]["B"] == pytest.approx(8.0)
    e = fit["parabola"]["band_branchfree_wins"]
    assert e[0] * (1 - e[0]) == pytest.approx((3.0 - 2.0) / 8.0)
    td = 1.0 + 4.0 * lawfit.p_div(s)
    fit = lawfit.fit_branch_models(s, td, np.full_like(s, 3.0))
    assert fit["divergence"]["A"] == pytest.approx(1.0) and fit["divergence"]["B"] == pytest.approx(4.0)
    # P_div: a group of 32 i.i.d. values is mixed with probability 1 - s^32 - (1-s)^32
    assert lawfit.p_div(0.5) == pytest.approx(1 - 2 * 0.5 ** 32)
    assert lawfit.p_div(0.0) == 0.0 and lawfit.p_div(1.0) == 0.0
    assert math.isclose(float(lawfit.p_div(0.01)), 1 - 0.01 ** 32 - 0.99 ** 32)
