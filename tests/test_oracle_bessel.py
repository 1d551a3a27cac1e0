"""Pins of the oracle's Bessel series (the thesis uses I_n throughout §3.2-§3.4)."""
import math

import numpy as np
import pytest
from scipy.special import iv

from oracle import bessel_i


@pytest.mark.parametrize("x", [1e-6, 0.05, 0.3, 1.0, 1.6, 2.0, 3.7, 8.0])
@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 9, 17, 40])
def test_series_matches_library(n, x):
    ref = iv(n, x)
    got = bessel_i(n, x)
    if ref < 1e-300:
        assert got < 1e-290
    elif ref < 1e-290:
        assert abs(got / ref - 1.0) < 1e-12  # subnormal-adjacent range
    else:
        assert abs(got / ref - 1.0) < 2e-14
    assert bessel_i(-n, x) == got


@pytest.mark.parametrize("n,x", [(0, 1.3), (2, 0.7), (4, 2.2), (7, 1.1)])
def test_series_matches_trapezoid_integral(n, x):
    # I_n(x) = (1/pi) int_0^pi exp(x cos t) cos(n t) dt; periodic analytic integrand,
    # so the full-period trapezoid rule converges geometrically.
    Q = 128
    t = 2 * math.pi * np.arange(Q) / Q
    ref = float(np.mean(np.exp(x * np.cos(t)) * np.cos(n * t)))
    assert abs(bessel_i(n, x) - ref) < 1e-15 * max(1.0, abs(ref))


def test_generating_function_sum():
    # sum_n I_n(x) = exp(x) (generating function at t = 1)
    for x in [0.2, 1.0, 2.5]:
        s = sum(bessel_i(n, x) for n in range(-60, 61))
        assert abs(s / math.exp(x) - 1.0) < 1e-15


def test_zero_and_negative_argument():
    assert bessel_i(0, 0.0) == 1.0
    assert bessel_i(3, 0.0) == 0.0
    assert abs(bessel_i(3, -1.2) + bessel_i(3, 1.2)) < 1e-17
    assert bessel_i(2, -1.2) == bessel_i(2, 1.2)
