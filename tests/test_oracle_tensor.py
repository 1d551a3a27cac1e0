"""Pins of the gXY coefficients and site tensors (§3.2, §3.3, §3.4)."""
import math

import numpy as np
import pytest
from scipy.special import iv

from oracle import gxy
from oracle.bessel import bessel_i


def fourier_by_quadrature(beta, delta, n, Q=512):
    # a_n = (1/2pi) int e^{beta(Delta cos x + (1-Delta) cos 2x)} cos(n x) dx (Eq. 3.3 / 3.4)
    x = 2 * math.pi * np.arange(Q) / Q
    w = np.exp(beta * (delta * np.cos(x) + (1 - delta) * np.cos(2 * x)))
    return float(np.mean(w * np.cos(n * x)))


@pytest.mark.parametrize("beta,delta", [(1.0, 0.5), (1.6, 0.3), (1.0 / 0.694, 0.34), (2.0, 0.0), (0.5, 1.0), (1.1, 0.5)])
def test_coefficients_two_routes(beta, delta):
    a = gxy.fourier_coefficients(beta, delta, 6)
    for n in range(-6, 7):
        ref = fourier_by_quadrature(beta, delta, n)
        assert abs(a[n + 6] - ref) < 1e-15 * max(1.0, abs(ref)) * 8


def test_coefficients_special_cases():
    beta = 1.3
    # Delta = 1: plain XY, a_n = I_n(beta)
    a = gxy.fourier_coefficients(beta, 1.0, 5)
    for n in range(-5, 6):
        assert abs(a[n + 5] - iv(n, beta)) < 1e-15 * iv(0, beta)
    # Delta = 0: pure nematic, a_{2k} = I_k(beta), a_odd = 0
    a = gxy.fourier_coefficients(beta, 0.0, 6)
    for n in range(-6, 7):
        ref = iv(n // 2, beta) if n % 2 == 0 else 0.0
        assert abs(a[n + 6] - ref) < 1e-15 * iv(0, beta)
    # sum_n a_n = w(0) = exp(beta) (the bond weight at zero angle)
    a = gxy.fourier_coefficients(0.9, 0.37, 40)
    assert abs(a.sum() / math.exp(0.9) - 1.0) < 1e-14
    # a_{-n} = a_n
    assert np.allclose(a, a[::-1], rtol=1e-14, atol=0)


def test_site_tensor_charge_rule_and_values():
    beta, delta, nm = 1.1, 0.5, 3
    a = gxy.fourier_coefficients(beta, delta, nm)
    T = gxy.site_tensor(beta, delta, nm)
    D0 = 2 * nm + 1
    for l in range(D0):
        for r in range(D0):
            for u in range(D0):
                for d in range(D0):
                    if l + u == r + d:
                        assert T[l, r, u, d] == pytest.approx(math.sqrt(a[l] * a[r] * a[u] * a[d]), rel=1e-15)
                    else:
                        assert T[l, r, u, d] == 0.0


def field_by_quadrature(Q, beta, h, h1, insert=None, n=256):
    t = 2 * math.pi * np.arange(n) / n
    g = np.exp(beta * h * np.cos(t) + beta * h1 * np.cos(2 * t))
    if insert is not None:
        g = g * insert(t)
    return float(np.mean(g * np.cos(Q * t)))


@pytest.mark.parametrize("h,h1", [(0.0, 0.0), (0.05, 0.0), (0.0, 0.04), (0.3, 0.2)])
def test_field_and_impurity_factors(h, h1):
    beta = 1.2
    for Q in range(-5, 6):
        f = gxy.field_factor(Q, beta, h, h1, gxy.PURE)
        assert abs(f - field_by_quadrature(Q, beta, h, h1)) < 1e-15
        fm = gxy.field_factor(Q, beta, h, h1, gxy.IMP_M)
        assert abs(fm - field_by_quadrature(Q, beta, h, h1, np.cos)) < 1e-15
        fm1 = gxy.field_factor(Q, beta, h, h1, gxy.IMP_M1)
        assert abs(fm1 - field_by_quadrature(Q, beta, h, h1, lambda t: np.cos(2 * t))) < 1e-15
    if h == 0.0 and h1 == 0.0:
        assert gxy.field_factor(0, beta, 0, 0) == 1.0
        assert gxy.field_factor(2, beta, 0, 0) == 0.0


def test_ising_tensor_bond_weights():
    b = 0.37
    T = gxy.ising_tensor(b)
    # parity rule and full symmetry under leg permutations
    for idx in np.ndindex(2, 2, 2, 2):
        if sum(idx) % 2:
            assert abs(T[idx]) < 1e-15
    assert np.allclose(T, T.transpose(1, 0, 3, 2)) and np.allclose(T, T.transpose(2, 3, 0, 1))
    # a 1x1 periodic closure = sum_s exp(2 b) (two self-bonds) = 2 e^{2b}
    assert abs(np.einsum("xxyy->", T) - 2 * math.exp(2 * b)) < 1e-13
