"""Pins of the phase-boundary oracle (peaks, parabolic refinement, zero-field fit).

Each part is checked against something other than itself: scipy.signal's
find_peaks (local maxima with plateaus, prominences), exact quadratics (the
three-point vertex is exact on them), scipy.optimize.curve_fit (a
Levenberg-Marquardt solver, not the profile root the oracle takes), ordinary
linear regression (the c = 1 case), and exact synthetic data.
"""
import math

import numpy as np
import pytest
from scipy import optimize, signal

from oracle import observables as OO
from oracle import phase as OP


@pytest.mark.parametrize("seed", range(6))
def test_local_maxima_and_prominences_match_scipy(seed):
    rng = np.random.default_rng(seed)
    # a quantised random walk has plateaus, equal neighbours and ties at the ends
    y = np.round(np.cumsum(rng.standard_normal(300)) * 2) / 2
    idx = OP.local_maxima(y)
    ref, _ = signal.find_peaks(y)
    assert idx == list(ref)
    pr = [OP.prominence(list(y), p) for p in idx]
    ref_pr = signal.peak_prominences(y, ref)[0]
    assert np.array_equal(np.array(pr), ref_pr)
    thr = float(np.median(ref_pr))
    kept = [p for p, q in zip(idx, pr) if q >= thr]
    assert kept == list(signal.find_peaks(y, prominence=thr)[0])


def test_no_peak_cases():
    assert OP.local_maxima([]) == [] and OP.local_maxima([1.0]) == [] and OP.local_maxima([1.0, 2.0]) == []
    assert OP.local_maxima([1.0, 2.0, 3.0]) == []  # monotone: the end is not a peak
    assert OP.local_maxima([2.0, 2.0, 2.0, 2.0]) == []  # flat
    assert OP.local_maxima([0.0, 1.0, 1.0, 1.0, 1.0, 0.0]) == [2]  # plateau: its middle (scipy's rule)
    assert OP.find_peaks([0.0, 1.0, 2.0], [3.0, 2.0, 1.0]) == []
    # a plateau of four samples: the flat window's peak is its middle sample; of two: between them
    assert OP.find_peaks([0.0, 1.0, 2.0, 3.0, 4.0, 5.0], [0.0, 1.0, 1.0, 1.0, 1.0, 0.0]) == [(2.0, 1.0, 1.0)]
    (xv, yv, pr), = OP.find_peaks([0.0, 1.0, 2.0, 3.0], [0.0, 1.0, 1.0, 0.0])
    assert abs(xv - 1.5) < 1e-15 and abs(yv - 1.125) < 1e-15 and pr == 1.0


def test_vertex_is_exact_on_quadratics():
    rng = np.random.default_rng(3)
    for _ in range(50):
        A = -rng.uniform(0.5, 20.0)
        x0 = rng.uniform(0.6, 1.4)
        y0 = rng.uniform(-1, 5)
        x = np.sort(x0 + rng.uniform(-0.05, 0.05, 3))
        y = A * (x - x0) ** 2 + y0
        xv, yv = OP.vertex(x, y)
        assert abs(xv - x0) <= 1e-11 and abs(yv - y0) <= 1e-11 * max(1.0, abs(y0))
    # symmetric samples put the vertex on the middle point
    xv, _ = OP.vertex([0.9, 1.0, 1.1], [2.0, 3.0, 2.0])
    assert abs(xv - 1.0) <= 1e-15


def test_find_peaks_two_branches_and_cap():
    # max of two parabolas: every 3-point window around a peak lies on one branch,
    # so both refined peaks are exact; the cap keeps the more prominent one
    x = np.linspace(0.0, 1.0, 41) ** 1.1  # non-uniform grid
    y = np.maximum(-30 * (x - 0.31) ** 2 + 1.0, -50 * (x - 0.77) ** 2 + 1.4)
    pk = OP.find_peaks(x, y)
    assert len(pk) == 2
    assert abs(pk[0][0] - 0.31) < 1e-11 and abs(pk[0][1] - 1.0) < 1e-11
    assert abs(pk[1][0] - 0.77) < 1e-11 and abs(pk[1][1] - 1.4) < 1e-11
    one = OP.find_peaks(x, y, cap=1)
    assert len(one) == 1 and abs(one[0][0] - 0.77) < 1e-11
    assert OP.find_peaks(x, y, min_prominence=10.0) == []
    # prominence of the lower peak: its height above the kink between the branches
    assert OP.find_peaks(x, y)[0][2] < OP.find_peaks(x, y)[1][2]


H_BAR = np.array([0.005, 0.01, 0.015, 0.02, 0.03, 0.04, 0.05])


def test_fit_recovers_exact_data():
    # the fit parameters the thesis prints for Delta = 0.32, as a realistic instance
    a, b, c = 0.685, 0.48, 0.29
    f = OP.fit_tc(H_BAR, a + b * H_BAR ** c)
    assert abs(f["a"] - a) < 1e-10 and abs(f["b"] - b) < 1e-10 and abs(f["c"] - c) < 1e-10
    assert f["rss"] < 1e-24 and f["at_bound"] == 0 and f["n"] == len(H_BAR)
    # three points determine the curve: zero errors by definition
    g = OP.fit_tc(H_BAR[:3], a + b * H_BAR[:3] ** c)
    assert abs(g["a"] - a) < 1e-8 and g["a_err"] == 0.0


@pytest.mark.parametrize("seed", range(4))
def test_fit_matches_curve_fit_on_noisy_data(seed):
    rng = np.random.default_rng(seed)
    a, b, c = 0.74, 0.9, 0.45
    t = a + b * H_BAR ** c + 2e-3 * rng.standard_normal(len(H_BAR))
    f = OP.fit_tc(H_BAR, t)
    p, pcov = optimize.curve_fit(lambda h, A, B, C: A + B * h ** C, H_BAR, t, p0=[f["a"] + 0.01, f["b"] * 1.1,
                                                                                 f["c"] * 0.9],
                                 method="lm", xtol=1e-15, ftol=1e-15, maxfev=100000)
    assert np.allclose([f["a"], f["b"], f["c"]], p, rtol=1e-7, atol=1e-9)
    assert np.allclose([f["a_err"], f["b_err"], f["c_err"]], np.sqrt(np.diag(pcov)), rtol=1e-5)
    # and it is a minimum of the residual sum over a brute-force neighbourhood
    def rss(A, B, C):
        return float(np.sum((t - A - B * H_BAR ** C) ** 2))
    base = rss(f["a"], f["b"], f["c"])
    assert abs(base - f["rss"]) <= 1e-12 * base
    for d in rng.standard_normal((200, 3)) * 1e-4:
        assert rss(f["a"] + d[0], f["b"] + d[1], f["c"] + d[2]) >= base


def test_fit_c_one_is_linear_regression():
    rng = np.random.default_rng(7)
    t = 0.8 + 1.7 * H_BAR + 1e-4 * rng.standard_normal(len(H_BAR))
    f = OP.fit_tc(H_BAR, t, c_lo=1.0, c_hi=1.0)
    slope, icpt = np.polyfit(H_BAR, t, 1)
    assert f["at_bound"] == 1
    assert abs(f["a"] - icpt) < 1e-12 and abs(f["b"] - slope) < 1e-10


def test_fit_minimum_on_a_bound():
    t = 0.7 + 50.0 * H_BAR ** 3.0  # true exponent above the bracket [0.05, 2]
    f = OP.fit_tc(H_BAR, t)
    assert f["at_bound"] == 1 and f["c"] == OP.C_HI


def test_fit_rejects_bad_input():
    with pytest.raises(ValueError):
        OP.fit_tc([0.01, 0.02], [0.8, 0.81])
    with pytest.raises(ValueError):
        OP.fit_tc([0.0, 0.01, 0.02], [0.8, 0.81, 0.82])
    with pytest.raises(ValueError):
        OP.fit_tc(H_BAR, H_BAR, c_lo=1.0, c_hi=0.5)


def test_field_rule():
    assert OP.field_for(0.36) == OP.FIELD_M1 and OP.field_for(0.37) == OP.FIELD_M
    assert OP.field_for(0.2, OP.FIELD_M) == OP.FIELD_M


def test_scans_compose_the_observables():
    temps = [0.9, 1.1]
    chi = OP.chi_scan(0.8, 2, 8, 6, temps, [0.02], dh=1e-3)
    assert chi.shape == (1, 2)
    assert chi[0, 1] == OO.susceptibility(1 / 1.1, 0.8, 2, 8, 6, 0.02, 1e-3, "h")
    cv = OP.cv_scan(0.8, 2, 8, 6, temps)
    assert cv[0] == OO.specific_heat(1 / 0.9, 0.8, 2, 8, 6)[0]


def test_tiny_scan_moves_the_peak_with_the_field():
    # D_cut = 8, 10 steps: an interior chi peak at every field, moving up in T with hbar
    temps = np.linspace(0.8, 1.4, 13)
    hbars = [0.01, 0.02, 0.04]
    chi = OP.chi_scan(0.8, 2, 8, 10, temps, hbars)
    tp = [OP.chi_peak(temps, row) for row in chi]
    assert all(not math.isnan(v) for v in tp)
    assert tp[0] < tp[1] < tp[2]
    f = OP.fit_tc(hbars, tp)
    assert f["a"] < tp[0] and f["b"] > 0


def test_ising_cv_matches_onsager_and_its_peak_locates_tc():
    # The 2D Ising model is solved exactly (Onsager): away from T_c the C_V difference
    # quotient of the HOTRG oracle equals that of the exact ln Z / N, and the refined C_V
    # peak of a temperature scan sits at T_c = 2 / ln(1 + sqrt 2) to well within the grid
    # spacing (the lattice of 2^24 sites and D_cut = 12 shift it by ~3e-4).
    from oracle import exact, gxy
    from oracle import hotrg as OH
    hb = 1e-2

    def cv_of(lnz_fn, T):
        b = 1.0 / T
        return b * b * (lnz_fn(b + hb) - 2.0 * lnz_fn(b) + lnz_fn(b - hb)) / hb ** 2

    def hotrg_lnz(steps, dcut):
        return lambda b: OH.hotrg_run(gxy.ising_tensor(b), gxy.ising_charges(), steps, dcut, "z2").lnz_per_site

    for T in (1.8, 3.0):
        assert abs(cv_of(hotrg_lnz(24, 16), T) - cv_of(exact.onsager_lnz, T)) < 1e-5
    tc = 2.0 / math.log(1.0 + math.sqrt(2.0))
    temps = np.linspace(2.22, 2.32, 11)
    cv = [cv_of(hotrg_lnz(24, 12), T) for T in temps]
    (t_peak, _, _), = OP.find_peaks(temps, cv, min_prominence=0.1)
    assert abs(t_peak - tc) < 2e-3
