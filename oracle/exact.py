"""Exact references that pin the oracle to something other than itself.

TEST INFRASTRUCTURE (oracle).  None of these routines uses the HOTRG code:

* ``tensor_network_lnz``: the tensor trace tTr of §2.4.1 / Eq. 3.16 on a small
  periodic Lx x Ly lattice, by the row-to-row transfer matrix
  R[(u_1..u_Lx),(d_1..d_Lx)] = sum_h prod_s T[h_{s-1}, h_s, u_s, d_s]
  (h_0 = h_Lx), Z = Tr R^Ly.
* ``direct_integral_lnz``: the partition function of §3.2 (Eq. 3.2) written as
  an integral over the angles, with the bond weight truncated to its
  Fourier modes |n| <= n_max, w(x) = a_0 + 2 sum_{n>=1} a_n cos(nx), and the
  on-site field factor exp(beta h cos t + beta h1 cos 2t) of Eq. 3.7.  The
  Q-point product trapezoid rule is exact for trigonometric polynomials of
  degree < Q in each angle, so with h = h1 = 0 and Q > 4 n_max it equals the
  tensor trace to rounding; with a field it converges exponentially in Q.
* ``onsager_lnz``: Onsager's closed form for the 2D Ising model.
* ``high_temperature_lnz``: the leading terms of the small-beta expansion,
  ln Z/N = 2 ln a_0 + sum_{n != 0} (a_n / a_0)^4 + O(u^6), u = max (a_n/a_0).
"""

import math

import numpy as np
from scipy import integrate


def tensor_network_lnz(T, Lx, Ly):
    """ln Z of the periodic Lx x Ly network of identical site tensors T[l,r,u,d]."""
    D = T.shape[0]
    Dv = T.shape[2]
    # X[h0, h, U, Dn] accumulated site by site along the row
    X = T.copy()  # (h0, h1, u1, d1)
    for _ in range(1, Lx):
        # X[h0,h,U,Dn] * T[h,h',u,d] -> X[h0,h',(U,u),(Dn,d)]
        X = np.einsum("ahUV,hbud->abUuVd", X, T)
        a, b, U, u, V, d = X.shape
        X = X.reshape(a, b, U * u, V * d)
    R = np.einsum("aaUV->UV", X)  # periodic horizontal closure
    assert R.shape == (Dv ** Lx, Dv ** Lx) and D == T.shape[1]
    M = np.linalg.matrix_power(R, Ly)
    return math.log(np.trace(M))


def bond_weight(x, a, n_max):
    """Truncated bond weight a_0 + 2 sum_{n=1}^{n_max} a_n cos(n x); a indexed n + n_max."""
    w = np.full_like(x, a[n_max])
    for n in range(1, n_max + 1):
        w = w + 2.0 * a[n_max + n] * np.cos(n * x)
    return w


def direct_integral_lnz(a, n_max, Lx, Ly, Q, beta=0.0, h=0.0, h1=0.0, insert=None):
    """ln Z (and optionally <insert(theta_0)>) of the periodic Lx x Ly lattice.

    a: Fourier coefficients indexed n + n_max.  Angle-space transfer matrix
    K[(t_1..t_Lx), (t'_1..t'_Lx)] = prod_s g(t_s)/Q * w(t_s - t_{s+1}) * w(t_s - t'_s),
    Z = Tr K^Ly.  ``insert`` (a function of one angle) returns
    (ln Z, <insert(theta)> at one site).
    """
    th = 2.0 * math.pi * np.arange(Q) / Q
    g = np.exp(beta * h * np.cos(th) + beta * h1 * np.cos(2.0 * th)) / Q
    W = bond_weight(th[:, None] - th[None, :], a, n_max)  # W[t, t']
    grids = np.meshgrid(*([np.arange(Q)] * Lx), indexing="ij")
    idx = [gg.reshape(-1) for gg in grids]  # configuration -> angle index per site
    n = Q ** Lx
    row = np.ones(n)
    for s in range(Lx):
        row = row * g[idx[s]] * W[idx[s], idx[(s + 1) % Lx]]
    K = row[:, None] * np.ones((1, n))
    for s in range(Lx):
        K = K * W[idx[s][:, None], idx[s][None, :]]
    M = np.linalg.matrix_power(K, Ly)
    Z = np.trace(M)
    if insert is None:
        return math.log(Z)
    ins = insert(th)[idx[0]]
    Zi = np.trace(M * ins[:, None])  # one insertion at site 0 of the first row
    return math.log(Z), Zi / Z


def onsager_lnz(beta):
    """ln Z / N of the infinite square-lattice Ising model (J = 1)."""
    k = 1.0 / math.sinh(2.0 * beta) ** 2
    c2 = math.cosh(2.0 * beta) ** 2

    def f(t):
        return math.log(c2 + math.sqrt(1.0 + k * k - 2.0 * k * math.cos(2.0 * t)) / k)

    val, _ = integrate.quad(f, 0.0, math.pi, epsabs=1e-14, epsrel=1e-14, limit=400,
                            points=[math.pi / 2.0])
    return 0.5 * math.log(2.0) + val / (2.0 * math.pi)


def high_temperature_lnz(a, n_max):
    """2 ln a_0 + sum_{n != 0} (a_n/a_0)^4 and the expansion parameter u."""
    a0 = a[n_max]
    r = np.array([a[n_max + n] / a0 for n in range(1, n_max + 1)])
    return 2.0 * math.log(a0) + 2.0 * float(np.sum(r ** 4)), float(np.max(np.abs(r)))
