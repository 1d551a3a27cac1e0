"""Pins of the oracle's HOTRG engine against exact and closed-form results.

* untruncated HOTRG on 2x2 and 4x4 periodic lattices = brute-force tensor trace
  = direct numerical integration of Z (§3.2, Eq. 3.2 / 3.16);
* truncated HOTRG on the 2D Ising tensor vs Onsager's closed form;
* Delta = 0 gXY == plain XY at half the charge cutoff (§3.1: Delta = 0 is the
  pure nematic model, an exact relabelling of the XY charges);
* the small-beta (high-temperature) series;
* the A/B regrouping of the environment == M_(l) M_(l)^T with M built as in Eq. 2.11.
"""
import math

import numpy as np
import pytest

from oracle import exact, gxy
from oracle import hotrg as H

UNTRUNC = 10 ** 9


@pytest.mark.parametrize("beta,delta,nm", [(1.0, 0.5, 1), (1.0, 0.5, 2), (1.7, 0.2, 2), (0.6, 0.9, 3), (1.2, 0.0, 2)])
def test_2x2_untruncated_exact(beta, delta, nm):
    T0 = gxy.site_tensor(beta, delta, nm)
    q = gxy.leg_charges(nm, "u1")
    r = H.hotrg_run(T0, q, 2, UNTRUNC)
    tn = exact.tensor_network_lnz(T0, 2, 2) / 4
    a = gxy.fourier_coefficients(beta, delta, nm)
    di = exact.direct_integral_lnz(a, nm, 2, 2, Q=4 * nm + 1) / 4
    assert abs(r.lnz_per_site - tn) < 1e-13 * max(1, abs(tn))
    assert abs(di - tn) < 1e-13 * max(1, abs(tn))
    # untruncated: nothing is discarded
    assert all(s.eps_left == pytest.approx(0, abs=1e-12) for s in r.steps)


def test_4x4_untruncated_exact():
    beta, delta, nm = 1.0, 0.5, 1
    T0 = gxy.site_tensor(beta, delta, nm)
    r = H.hotrg_run(T0, gxy.leg_charges(nm, "u1"), 4, UNTRUNC)
    tn = exact.tensor_network_lnz(T0, 4, 4) / 16
    di = exact.direct_integral_lnz(gxy.fourier_coefficients(beta, delta, nm), nm, 4, 4, Q=5) / 16
    assert abs(r.lnz_per_site - tn) < 1e-13
    assert abs(di - tn) < 1e-13


@pytest.mark.parametrize("h,h1", [(0.0, 0.08), (0.1, 0.0), (0.07, 0.05)])
def test_2x2_with_fields_and_impurities(h, h1):
    beta, delta, nm = 1.1, 0.4, 2
    sym = gxy.symmetry_of(h, h1)
    T0 = gxy.site_tensor(beta, delta, nm, h, h1)
    q = gxy.leg_charges(nm, sym)
    a = gxy.fourier_coefficients(beta, delta, nm)
    r = H.hotrg_run(T0, q, 2, UNTRUNC, sym)
    tn = exact.tensor_network_lnz(T0, 2, 2) / 4
    assert abs(r.lnz_per_site - tn) < 1e-13
    # the field factor is not a trig polynomial: Q = 48 converges to rounding here
    lz, mcos = exact.direct_integral_lnz(a, nm, 2, 2, 48, beta, h, h1, insert=np.cos)
    assert abs(lz / 4 - tn) < 1e-13
    lz, mcos2 = exact.direct_integral_lnz(a, nm, 2, 2, 48, beta, h, h1, insert=lambda t: np.cos(2 * t))
    Ti = gxy.site_tensor(beta, delta, nm, h, h1, gxy.IMP_M)
    rm = H.hotrg_run(T0, q, 2, UNTRUNC, sym, T_imp0=Ti)
    assert abs(rm.imp_ratio - mcos) < 1e-13
    Ti1 = gxy.site_tensor(beta, delta, nm, h, h1, gxy.IMP_M1)
    rm1 = H.hotrg_run(T0, q, 2, UNTRUNC, sym, T_imp0=Ti1)
    assert abs(rm1.imp_ratio - mcos2) < 1e-13


def test_onsager_closed_form_itself():
    # high-temperature limit ln 2, low-temperature limit 2 beta, and the exact
    # critical value ln2/2 + 2G/pi (G = Catalan's constant)
    assert abs(exact.onsager_lnz(1e-4) - math.log(2)) < 1e-7
    assert abs(exact.onsager_lnz(6.0) - 12.0) < 1e-9
    bc = 0.5 * math.log(1 + math.sqrt(2))
    catalan = 0.915965594177219015054603514932384110774
    assert abs(exact.onsager_lnz(bc) - (0.5 * math.log(2) + 2 * catalan / math.pi)) < 1e-12


@pytest.mark.parametrize("beta,tol", [(0.3, 1e-9), (0.6, 1e-9), (0.4406868, 1e-6)])
def test_ising_vs_onsager(beta, tol):
    r = H.hotrg_run(gxy.ising_tensor(beta), gxy.ising_charges(), 30, 16, "z2")
    assert abs(r.lnz_per_site - exact.onsager_lnz(beta)) < tol


def test_delta0_maps_onto_xy():
    beta = 1.3
    g = H.run_gxy(beta, 0.0, 4, 12, 16)   # gXY, Delta = 0, n_max = 2K
    x = H.run_gxy(beta, 1.0, 2, 12, 16)   # XY (Delta = 1), n_max = K
    assert abs(g.lnz_per_site - x.lnz_per_site) < 1e-14


@pytest.mark.parametrize("beta", [0.05, 0.1])
def test_high_temperature_series(beta):
    a = gxy.fourier_coefficients(beta, 0.5, 2)
    ht, u = exact.high_temperature_lnz(a, 2)
    r = H.run_gxy(beta, 0.5, 2, 16, 20)
    assert abs(r.lnz_per_site - ht) <= 10 * u ** 6


def test_environment_regrouping_matches_definition():
    rng = np.random.default_rng(7)
    Dh, Dv = 3, 4
    T = rng.standard_normal((Dh, Dh, Dv, Dv))
    # Eq. 2.11: M[(l1,l2),(r1,r2),u,d] = sum_i T[l1,r1,u,i] T[l2,r2,i,d]
    M = np.einsum("aeui,bfid->abefud", T, T)
    ML = M.reshape(Dh * Dh, -1)
    assert np.allclose(H.environment_left(T), ML @ ML.T, rtol=1e-13, atol=1e-12)
    MR = M.transpose(2, 3, 0, 1, 4, 5).reshape(Dh * Dh, -1)
    assert np.allclose(H.environment_right(T), MR @ MR.T, rtol=1e-13, atol=1e-12)
    # the coarse tensor (Eq. 2.16) against P^T M P with M explicit
    P = np.linalg.qr(rng.standard_normal((Dh * Dh, 5)))[0]
    Tn = H.coarse(P.reshape(Dh, Dh, 5), T, T)
    ref = np.einsum("ax,abud,by->xyud", P, M.reshape(Dh * Dh, Dh * Dh, Dv, Dv), P)
    assert np.allclose(Tn, ref, rtol=1e-13, atol=1e-12)


def test_sector_eigensolve_equals_dense():
    beta, delta, nm = 1.2, 0.5, 2
    T0 = gxy.site_tensor(beta, delta, nm)
    T0 = T0 / np.linalg.norm(T0)
    q = gxy.leg_charges(nm, "u1")
    E = H.environment_left(T0)
    cands = H.sector_eigen(E, H.fused_charges(q, "u1"))
    lam = np.sort([c[0] for c in cands])
    assert np.allclose(lam, np.linalg.eigvalsh(E), atol=1e-14)
    # E is block diagonal in the fused charge
    qf = H.fused_charges(q, "u1")
    assert np.all(E[qf[:, None] != qf[None, :]] == 0.0)


def test_cut_cluster_rule():
    # equal eigenvalues in sectors +1/-1 at the cut: +q is kept first, then larger lambda
    v = np.zeros(4)
    cands = [(1.0, 0, 0, v), (0.5, 1, 0, v), (0.5, -1, 0, v), (0.5 + 1e-15, 2, 0, v), (0.1, 0, 1, v)]
    keep = H.select_kept(cands, 2)
    assert keep == [0, 1]
    keep = H.select_kept(cands, 3)
    assert keep == [0, 1, 2]
    keep = H.select_kept(cands, 4)
    assert keep == [0, 1, 2, 3]


def test_gauge_invariants_do_not_depend_on_side_policy_untruncated():
    r0 = H.run_gxy(1.0, 0.5, 1, 81, 3, env_policy=0)
    r1 = H.run_gxy(1.0, 0.5, 1, 81, 3, env_policy=1)
    assert abs(r0.lnz_per_site - r1.lnz_per_site) < 1e-14
