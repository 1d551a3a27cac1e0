"""Initial tensors of the q = 2 generalized XY model (and the 2D Ising pin).

The order q of the second coupling is a parameter (default 2, the thesis's
model); only the coefficients a_n depend on it.

TEST INFRASTRUCTURE (oracle).  Follows §3.2-§3.4 of the thesis:

* Fourier / character coefficients (§3.2, Eq. 3.4):
      a_n(beta, Delta) = sum_m I_{n-2m}(beta Delta) I_m(beta (1 - Delta)),
  with the infinite sum truncated to m in [-50, 50] as the thesis does (§3.2).
  The bond weight exp(beta[Delta cos x + (1-Delta) cos 2x]) equals
  sum_n a_n e^{inx}; these a_n are the t_n of the site tensor.
* Site tensor (§3.2, Eq. 3.6; §3.3, Eq. 3.15):
      T[l,r,u,d] = sqrt(a_l a_r a_u a_d) * F(Q),
      F(Q) = sum_j I_{Q+2j}(beta h) I_j(beta h1),   Q = n_l + n_u - n_r - n_d,
  with leg index i <-> charge n = i - n_max (D0 = 2 n_max + 1 states).  At
  h = h1 = 0, F(Q) = delta_{Q,0}: the U(1) rule n_l + n_u = n_r + n_d.
  (The thesis labels the legs top/right/bottom/left with n1+n2-n3-n4; the
  rule used here is that one with up and down exchanged, a reflection of the
  lattice, and F(-Q) = F(Q), so Z is unchanged.)
* Impurity tensors for <cos theta> and <cos 2 theta> (§3.4, Eq. 3.20, 3.21):
  F is replaced by
      F_M(Q)  = sum_j I_j(beta h1) [I_{Q+2j-1}(beta h) + I_{Q+2j+1}(beta h)] / 2
      F_M1(Q) = sum_j I_{Q+2j}(beta h) [I_{j+1}(beta h1) + I_{j-1}(beta h1)] / 2
  The thesis's definition M = (1/beta) d ln Z / dh makes P / Z with this
  impurity the per-site magnetisation <cos theta>.
* 2D Ising tensor (pin for the HOTRG engine against Onsager): with
  W = [[sqrt(cosh b), sqrt(sinh b)], [sqrt(cosh b), -sqrt(sinh b)]],
  T[l,r,u,d] = sum_s W[s,l] W[s,r] W[s,u] W[s,d]; each bond gives
  sum_k W[s,k] W[s',k] = exp(b s s').

Symmetry labels: ``sym`` is "u1" (h = h1 = 0: charge conserved), "z2"
(h = 0, h1 != 0: charge parity conserved; also the Ising tensor) or "none"
(h != 0).  They only select the block structure used by the eigensolve.
"""

import math

import numpy as np

from .bessel import bessel_i

M_RANGE = 50  # the thesis's truncation m in [-50, 50] (§3.2)

# tensor kinds
PURE, IMP_M, IMP_M1 = "pure", "imp_m", "imp_m1"


def fourier_coefficients(beta: float, delta: float, n_max: int, m_range: int = M_RANGE, q: int = 2):
    """a_n for n = -n_max..n_max (index n + n_max), §3.2 Eq. 3.4.

    q is the order of the second coupling, cos(q x): the thesis's model is
    q = 2; the q >= 3 generalisations it names as future work (§4, §6) change
    only these coefficients, a_n = sum_m I_{n - q m}(beta Delta) I_m(beta (1 - Delta)).
    """
    x1 = beta * delta
    x2 = beta * (1.0 - delta)
    out = np.zeros(2 * n_max + 1)
    for n in range(-n_max, n_max + 1):
        s = 0.0
        for m in range(-m_range, m_range + 1):
            s += bessel_i(n - q * m, x1) * bessel_i(m, x2)
        out[n + n_max] = s
    return out


def field_factor(Q: int, beta: float, h: float, h1: float, kind: str = PURE,
                 m_range: int = M_RANGE) -> float:
    """Charge-imbalance factor of the site tensor (Eq. 3.15, 3.20, 3.21)."""
    bh = beta * h
    bh1 = beta * h1
    s = 0.0
    for j in range(-m_range, m_range + 1):
        if kind == PURE:
            s += bessel_i(Q + 2 * j, bh) * bessel_i(j, bh1)
        elif kind == IMP_M:
            s += bessel_i(j, bh1) * 0.5 * (bessel_i(Q + 2 * j - 1, bh) + bessel_i(Q + 2 * j + 1, bh))
        elif kind == IMP_M1:
            s += bessel_i(Q + 2 * j, bh) * 0.5 * (bessel_i(j + 1, bh1) + bessel_i(j - 1, bh1))
        else:
            raise ValueError(f"unknown tensor kind {kind!r}")
    return s


def symmetry_of(h: float, h1: float) -> str:
    """Block structure of the pure tensor: U(1) at zero field, Z2 with h1 only."""
    if h != 0.0:
        return "none"
    if h1 != 0.0:
        return "z2"
    return "u1"


def leg_charges(n_max: int, sym: str):
    """Integer labels of the D0 basis states of a bond (charge n = i - n_max)."""
    q = np.arange(-n_max, n_max + 1, dtype=np.int64)
    if sym == "z2":
        q = np.mod(q, 2)
    elif sym == "none":
        q = np.zeros_like(q)
    return q


def site_tensor(beta: float, delta: float, n_max: int, h: float = 0.0, h1: float = 0.0,
                kind: str = PURE, m_range: int = M_RANGE, q: int = 2):
    """T[l,r,u,d] of shape (D0,)*4, FP64 (Eq. 3.6 / 3.15 / 3.20 / 3.21); q as in fourier_coefficients."""
    a = fourier_coefficients(beta, delta, n_max, m_range, q)
    D0 = 2 * n_max + 1
    n = np.arange(-n_max, n_max + 1)
    fcache = {}
    T = np.zeros((D0, D0, D0, D0))
    for il in range(D0):
        for ir in range(D0):
            for iu in range(D0):
                for idn in range(D0):
                    Q = int(n[il] + n[iu] - n[ir] - n[idn])
                    if Q not in fcache:
                        fcache[Q] = field_factor(Q, beta, h, h1, kind, m_range)
                    f = fcache[Q]
                    if f == 0.0:
                        continue
                    T[il, ir, iu, idn] = math.sqrt(a[il] * a[ir] * a[iu] * a[idn]) * f
    return T


def ising_tensor(beta: float):
    """2D Ising site tensor with legs (l, r, u, d), bond dimension 2."""
    c = math.sqrt(math.cosh(beta))
    s = math.sqrt(math.sinh(beta))
    W = np.array([[c, s], [c, -s]])  # rows: spin +1, -1; columns: bond state 0, 1
    T = np.zeros((2, 2, 2, 2))
    for sp in range(2):
        T += np.einsum("a,b,c,d->abcd", W[sp], W[sp], W[sp], W[sp])
    return T


def ising_charges():
    """Z2 labels of the Ising bond states (the bond state is the parity)."""
    return np.array([0, 1], dtype=np.int64)
