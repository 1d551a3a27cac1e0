"""Host-only parts of the phase-boundary extraction (no device work): the
library's peak finder and zero-field fit against the oracle.

Peak positions (indices, prominences) are decisions and must be equal; the
refined vertex and the fit are floating point and agree to the rounding of
their two different routes (divided differences vs a Vandermonde solve;
false position vs brentq on the profile derivative)."""
import numpy as np
import pytest

from oracle import phase as OP


@pytest.fixture(scope="module")
def H():
    from paper_2609_20536_b300 import build
    build.build()
    from paper_2609_20536_b300 import hotrg
    return hotrg


def same_peaks(got, ref, xtol):
    assert len(got) == len(ref)
    for (x, y, p), (xr, yr, pr) in zip(got, ref):
        assert p == pr  # the same samples: exact
        assert abs(x - xr) <= xtol and abs(y - yr) <= 1e-12 * max(1.0, abs(yr))


@pytest.mark.parametrize("seed", range(8))
def test_peaks_match_oracle_on_random_curves(H, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 400))
    x = np.cumsum(rng.uniform(0.001, 0.02, n)) + 0.5
    y = np.round(np.cumsum(rng.standard_normal(n)) * 4) / 4  # plateaus of every length
    if seed % 2:
        y = np.sin(7 * x) + 1e-3 * rng.standard_normal(n)
    for thr, cap in ((0.0, 1000), (0.5, 1000), (0.0, 1), (0.25, 3)):
        got, nf = H.hotrg_find_peaks(x, y, thr, cap)
        ref = OP.find_peaks(x, y, thr, cap)
        assert nf == len(OP.find_peaks(x, y, thr))
        same_peaks(got, ref, 1e-12)


def test_peaks_edge_cases(H):
    assert H.hotrg_find_peaks([], [], 0.0, 4) == ([], 0)
    assert H.hotrg_find_peaks([1.0, 2.0], [0.0, 1.0], 0.0, 4) == ([], 0)
    assert H.hotrg_find_peaks([1.0, 2.0, 3.0], [1.0, 1.0, 1.0], 0.0, 4) == ([], 0)
    x = np.arange(6.0)
    got, nf = H.hotrg_find_peaks(x, [0.0, 1.0, 1.0, 1.0, 1.0, 0.0], 0.0, 4)
    assert nf == 1 and got == [(2.0, 1.0, 1.0)]  # flat window: the middle sample
    got, nf = H.hotrg_find_peaks(x[:4], [0.0, 1.0, 1.0, 0.0], 0.0, 4)
    assert nf == 1 and abs(got[0][0] - 1.5) < 1e-15 and abs(got[0][1] - 1.125) < 1e-15
    # cap 0: counts only
    got, nf = H.hotrg_find_peaks(x, [0.0, 2.0, 0.0, 1.0, 0.0, 0.0], 0.0, 0)
    assert got == [] and nf == 2
    for bad in (([0.0, 0.0, 1.0], [0.0, 1.0, 0.0]),   # not strictly ascending
                ([0.0, 1.0, 2.0], [0.0, np.nan, 0.0]),  # non-finite
                ([0.0, 2.0, 1.0], [0.0, 1.0, 0.0])):
        with pytest.raises(H.HotrgError):
            H.hotrg_find_peaks(*bad)
    with pytest.raises(H.HotrgError):
        H.hotrg_find_peaks([0.0, 1.0, 2.0], [0.0, 1.0, 0.0], float("inf"), 1)


HB = np.array([0.005, 0.01, 0.015, 0.02, 0.03, 0.04, 0.05])


def same_fit(f, r, tol=1e-9, etol=1e-6):
    assert f.n == r["n"] and f.at_bound == r["at_bound"]
    for k in ("a", "b", "c"):
        assert abs(getattr(f, k) - r[k]) <= tol * max(1.0, abs(r[k])), (k, getattr(f, k), r[k])
    for k in ("a_err", "b_err", "c_err"):
        assert abs(getattr(f, k) - r[k]) <= etol * max(abs(r[k]), 1e-300), (k, getattr(f, k), r[k])
    # exact data leave residuals at the rounding level of t ~ 1 (|r_i| ~ 1e-16)
    assert abs(f.rss - r["rss"]) <= 1e-9 * r["rss"] + 1e-24


@pytest.mark.parametrize("seed", range(6))
def test_fit_matches_oracle_on_noisy_data(H, seed):
    rng = np.random.default_rng(100 + seed)
    a, b, c = rng.uniform(0.6, 0.9), rng.uniform(0.2, 2.0), rng.uniform(0.15, 1.2)
    h = np.sort(rng.uniform(0.003, 0.06, int(rng.integers(4, 12))))
    t = a + b * h ** c + 1e-3 * rng.standard_normal(len(h))
    same_fit(H.hotrg_fit_tc(h, t), OP.fit_tc(h, t))


def test_fit_exact_and_three_points(H):
    t = 0.685 + 0.48 * HB ** 0.29
    f = H.hotrg_fit_tc(HB, t)
    assert abs(f.a - 0.685) < 1e-10 and abs(f.b - 0.48) < 1e-10 and abs(f.c - 0.29) < 1e-10
    g = H.hotrg_fit_tc(HB[:3], t[:3])
    assert g.n == 3 and g.a_err == 0.0 and abs(g.a - 0.685) < 1e-8
    same_fit(g, OP.fit_tc(HB[:3], t[:3]), tol=1e-8, etol=0.0)


def test_fit_bounds_and_fixed_exponent(H):
    t = 0.7 + 50.0 * HB ** 3.0
    f = H.hotrg_fit_tc(HB, t)
    same_fit(f, OP.fit_tc(HB, t))
    assert f.at_bound == 1 and f.c == 2.0
    rng = np.random.default_rng(7)
    t = 0.8 + 1.7 * HB + 1e-4 * rng.standard_normal(len(HB))
    f = H.hotrg_fit_tc(HB, t, 1.0, 1.0)
    same_fit(f, OP.fit_tc(HB, t, 1.0, 1.0))
    slope, icpt = np.polyfit(HB, t, 1)
    assert abs(f.a - icpt) < 1e-12 and abs(f.b - slope) < 1e-10
    # a minimum on the upper bound of an explicit bracket reports the bound exactly
    t = 0.7 + 50.0 * HB ** 3.0
    for hi in (1.7, 1.9, 2.3):
        f = H.hotrg_fit_tc(HB, t, 0.1, hi)
        assert f.at_bound == 1 and f.c == hi
    # a narrower bracket given explicitly
    t = 0.74 + 0.9 * HB ** 0.45 + 2e-3 * rng.standard_normal(len(HB))
    same_fit(H.hotrg_fit_tc(HB, t, 0.2, 0.8), OP.fit_tc(HB, t, 0.2, 0.8))


def test_fit_rejects_bad_input(H):
    for h, t, lo, hi in ((HB[:2], HB[:2], 0.0, 0.0),                  # too few points
                         ([0.01, 0.01, 0.02, 0.02], [0.8, 0.8, 0.81, 0.81], 0.0, 0.0),  # two distinct hbar
                         ([0.0, 0.01, 0.02], [0.8, 0.81, 0.82], 0.0, 0.0),
                         (HB, HB, 1.0, 0.5), (HB, HB, -1.0, 0.5),
                         (HB, np.where(HB > 0.02, np.nan, HB), 0.0, 0.0)):
        with pytest.raises(H.HotrgError):
            H.hotrg_fit_tc(h, t, lo, hi)


def test_cli_phase_summary_flags_truncation_artefacts(H):
    # a smooth C_V bump at T = 0.95 and an isolated dip to a negative value at T = 0.61,
    # the shape a change of the kept set between beta -+ hb leaves in the difference quotient
    import json
    from paper_2609_20536_b300.cli import phase_summary
    temps = np.linspace(0.55, 1.15, 41)
    cv = 2.2 - 8.0 * (temps - 0.95) ** 2
    cv[4] = -22.0
    fit = H.hotrg_fit_tc(HB[:4], 0.9 + 0.8 * HB[:4] ** 0.4)
    res = {"cv": cv, "t_peak": np.array([1.01, np.nan]), "fit": fit, "field": H.T_IMP_M, "status": 0}
    out = phase_summary(H, 0.8, 24, temps, [0.005, 0.04], res, 1.0)
    json.dumps(out)
    peaks = out["cv_peaks"]
    assert [p["next_to_negative_cv"] for p in peaks] == [True, False]
    assert abs(peaks[1]["T"] - 0.95) < 1e-12 and abs(peaks[1]["cv"] - 2.2) < 1e-12
    assert out["T_chi_peak"] == [1.01, None] and out["field"] == "h"
    assert abs(out["T_c_zero_field"] - 0.9) < 1e-9 and out["fit"]["n"] == 4
    # prominences 0.27 (the sample before the dip) and 0.32 (the bump): 0.3 keeps the bump; no fit gives null
    res["fit"] = H.TcFit()
    out = phase_summary(H, 0.8, 24, temps, [0.005, 0.04], res, 1.0, cv_prominence=0.3)
    assert len(out["cv_peaks"]) == 1 and out["fit"] is None and out["T_c_zero_field"] is None
