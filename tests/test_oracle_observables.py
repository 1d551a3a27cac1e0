"""Pins of the observables layer (§3.4, Eq. 3.17-3.21) and the Table 3.2 band."""
import math
import os

import numpy as np
import pytest

from oracle import exact, gxy
from oracle import hotrg as H
from oracle import observables as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_zero_field_magnetisation_vanishes():
    # U(1) symmetry at h = h1 = 0: one cos(theta) insertion has charge +-1, so P = 0
    m = O.magnetisation(1.2, 0.5, 2, 12, 10, 0.0, 0.0, gxy.IMP_M)
    assert abs(m) < 1e-15


def test_susceptibility_two_routes_exact_lattice():
    # 2x2 untruncated (exact): chi from the impurity m vs (1/beta) d^2 (lnZ/N) / dh^2
    beta, delta, nm, hb, dh = 1.1, 0.6, 2, 0.05, 1e-3

    def lnz(h):
        return H.run_gxy(beta, delta, nm, 10 ** 9, 2, h=h).lnz_per_site

    def m(h):
        return H.run_gxy(beta, delta, nm, 10 ** 9, 2, h=h, impurity=gxy.IMP_M).imp_ratio

    chi_imp = (m(hb + dh) - m(hb - dh)) / (2 * dh)
    chi_lnz = (lnz(hb + dh) - 2 * lnz(hb) + lnz(hb - dh)) / (beta * dh * dh)
    assert abs(chi_imp - chi_lnz) < 1e-5 * abs(chi_lnz)
    # and the first derivative: m = (1/beta) d (lnZ/N) / dh  (Eq. 3.19 per site)
    m_fd = (lnz(hb + dh) - lnz(hb - dh)) / (2 * dh * beta)
    assert abs(m(hb) - m_fd) < 1e-5 * abs(m_fd)  # central-difference error O(dh^2)


def test_specific_heat_step_halving():
    args = (1.0, 0.5, 2, 8, 12)
    c1, _ = O.specific_heat(*args, hb=1e-3)
    c2, _ = O.specific_heat(*args, hb=5e-4)
    assert abs(c1 - c2) < 1e-5 * abs(c1)


def test_specific_heat_exact_lattice_closed_form():
    # 2x2 untruncated: C_V against the analytic beta-derivative of the exact
    # direct integral, d^2 lnZ/dbeta^2 by a 5-point stencil (independent route)
    delta, nm, beta = 0.5, 1, 0.9

    def lnz_exact(b):
        a = gxy.fourier_coefficients(b, delta, nm)
        return exact.direct_integral_lnz(a, nm, 2, 2, 4 * nm + 1) / 4

    def lnz_hotrg(b):
        return H.run_gxy(b, delta, nm, 10 ** 9, 2).lnz_per_site

    hb = 1e-3
    cv = beta ** 2 * (lnz_hotrg(beta + hb) - 2 * lnz_hotrg(beta) + lnz_hotrg(beta - hb)) / hb ** 2
    h5 = 1e-2
    f = [lnz_exact(beta + k * h5) for k in (-2, -1, 0, 1, 2)]
    d2 = (-f[0] + 16 * f[1] - 30 * f[2] + 16 * f[3] - f[4]) / (12 * h5 * h5)
    assert abs(cv - beta ** 2 * d2) < 1e-6 * abs(cv)


def test_table_3_2_sanity_band():
    # F = -T lnZ/N at an unprinted h1 (Table 3.2).  At the oracle's small D the
    # printed F lies between the h1 = 0.01 and h1 = 0.03 values: a sanity band
    # for the sign and scale of the field term, not a parity pin.
    rows = np.loadtxt(os.path.join(GOLDEN, "table3_2_free_energy_m1.txt"))
    T = 0.694
    f_lo = -T * H.run_gxy(1 / T, 0.34, 4, 12, 24, h1=0.03).lnz_per_site
    f_hi = -T * H.run_gxy(1 / T, 0.34, 4, 12, 24, h1=0.01).lnz_per_site
    assert f_lo < rows[:, 1].min() and rows[:, 1].max() < f_hi
