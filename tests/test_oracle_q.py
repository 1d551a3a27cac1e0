"""The q >= 3 generalisation of the coupling cos(q theta) (the thesis's future
work): only the Fourier coefficients change.  Pins:

* q = 1: the weight is exp(beta cos x), so a_n = I_n(beta) for every Delta
  (the Bessel addition theorem sum_m I_{n-m}(x) I_m(y) = I_n(x + y));
* q = 3: a_n against the trapezoid Fourier integral of the bond weight, and
  Delta = 0 (weight exp(beta cos 3x)): a_{3k} = I_k(beta), others zero;
* the q = 3 site tensor on a 2 x 2 periodic lattice: untruncated HOTRG =
  brute-force tensor trace = direct angle integration of the truncated
  weight (exact trapezoid for a trigonometric polynomial).
"""
import math

import numpy as np
import pytest
from scipy import special

from oracle import exact, gxy
from oracle import hotrg as OH


@pytest.mark.parametrize("beta,delta", [(0.7, 0.2), (1.3, 0.9)])
def test_q1_reduces_to_xy(beta, delta):
    a = gxy.fourier_coefficients(beta, delta, 4, q=1)
    ref = np.array([special.iv(n, beta) for n in range(-4, 5)])
    np.testing.assert_allclose(a, ref, rtol=1e-13)


@pytest.mark.parametrize("beta,delta", [(0.8, 0.3), (1.5, 0.6)])
def test_q3_against_fourier_integral(beta, delta):
    a = gxy.fourier_coefficients(beta, delta, 5, q=3)
    Q = 256
    x = 2 * math.pi * np.arange(Q) / Q
    w = np.exp(beta * (delta * np.cos(x) + (1 - delta) * np.cos(3 * x)))
    ref = np.array([np.mean(w * np.cos(n * x)) for n in range(-5, 6)])
    np.testing.assert_allclose(a, ref, rtol=1e-12, atol=1e-15)


def test_q3_delta0():
    beta = 1.1
    a = gxy.fourier_coefficients(beta, 0.0, 6, q=3)
    for n in range(-6, 7):
        ref = special.iv(n // 3, beta) if n % 3 == 0 else 0.0
        assert abs(a[n + 6] - ref) <= 1e-14 * max(1.0, abs(ref))


def test_q3_two_by_two_lattice_three_routes():
    beta, delta, nm = 1.2, 0.4, 2
    T = gxy.site_tensor(beta, delta, nm, q=3)
    a = gxy.fourier_coefficients(beta, delta, nm, q=3)
    brute = exact.tensor_network_lnz(T, 2, 2) / 4
    direct = exact.direct_integral_lnz(a, nm, 2, 2, Q=4 * nm + 3) / 4
    hot = OH.run_gxy(beta, delta, nm, 10 ** 3, 2, q=3).lnz_per_site
    assert abs(brute - direct) < 1e-13 and abs(hot - brute) < 1e-13
    # and it differs from the q = 2 model
    assert abs(hot - OH.run_gxy(beta, delta, nm, 10 ** 3, 2).lnz_per_site) > 1e-3


@pytest.mark.parametrize("point", __import__("parity_points").Q_SHAPES)
def test_q_parity_points_are_well_conditioned(point):
    # as for the q = 2 points: rounding-level input noise (1e-15 for the FP64
    # form, 1e-10 for the split form) must move ln Z/N far below the tolerance
    beta, delta, nm, dcut, steps, q = point
    T0 = gxy.site_tensor(beta, delta, nm, q=q)
    q0 = gxy.leg_charges(nm, "u1")
    ref = OH.hotrg_run(T0, q0, steps, dcut, "u1").lnz_per_site
    for eta, bound in ((1e-15, 2e-12), (1e-10, 2e-10)):
        rng = np.random.default_rng(3)
        Tp = T0 * (1.0 + eta * rng.standard_normal(T0.shape))
        assert abs(OH.hotrg_run(Tp, q0, steps, dcut, "u1").lnz_per_site - ref) <= bound
