"""Thermodynamic observables from HOTRG (§3.4 of the thesis).

TEST INFRASTRUCTURE (oracle).

* f = -T ln Z / N = -(ln Z / N) / beta (the F of §3.4, per site).
* Specific heat, Eq. 3.17: C_V = beta^2 / V d^2 ln Z / d beta^2, by the
  3-point central difference with step hb (1e-3 by default).
* Magnetisation, Eq. 3.19 with the impurity method of §3.4: per site
  m = P / Z = <cos theta> with the impurity tensor of Eq. 3.20, and
  m1 = <cos 2 theta> with Eq. 3.21.
* Susceptibility, Eq. 3.18, by a central finite difference of m in the field:
  chi = [m(hbar + dh) - m(hbar - dh)] / (2 dh)  (chi1 likewise with m1, h1).
  The thesis prints neither hbar nor dh ("parity unpinned" for those values);
  the formula is pinned by the second route d^2 (ln Z/N) / (beta dh^2).
"""

from dataclasses import dataclass

from . import gxy
from .hotrg import run_gxy


@dataclass
class Observables:
    lnz: float
    f: float
    cv: float
    m: float
    m1: float
    chi: float
    chi1: float


def lnz(beta, delta, n_max, d_cut, n_steps, h=0.0, h1=0.0, env_policy=0):
    return run_gxy(beta, delta, n_max, d_cut, n_steps, h, h1, env_policy).lnz_per_site


def specific_heat(beta, delta, n_max, d_cut, n_steps, hb=1e-3, h=0.0, h1=0.0, env_policy=0):
    lp = lnz(beta + hb, delta, n_max, d_cut, n_steps, h, h1, env_policy)
    l0 = lnz(beta, delta, n_max, d_cut, n_steps, h, h1, env_policy)
    lm = lnz(beta - hb, delta, n_max, d_cut, n_steps, h, h1, env_policy)
    return beta * beta * (lp - 2.0 * l0 + lm) / (hb * hb), l0


def magnetisation(beta, delta, n_max, d_cut, n_steps, h=0.0, h1=0.0, kind=gxy.IMP_M, env_policy=0):
    r = run_gxy(beta, delta, n_max, d_cut, n_steps, h, h1, env_policy, impurity=kind)
    return r.imp_ratio


def susceptibility(beta, delta, n_max, d_cut, n_steps, hbar, dh, which="h", env_policy=0):
    """chi = dm/dh (which='h', m = <cos t>) or chi1 = dm1/dh1 (which='h1')."""
    if which == "h":
        mp = magnetisation(beta, delta, n_max, d_cut, n_steps, hbar + dh, 0.0, gxy.IMP_M, env_policy)
        mm = magnetisation(beta, delta, n_max, d_cut, n_steps, hbar - dh, 0.0, gxy.IMP_M, env_policy)
    else:
        mp = magnetisation(beta, delta, n_max, d_cut, n_steps, 0.0, hbar + dh, gxy.IMP_M1, env_policy)
        mm = magnetisation(beta, delta, n_max, d_cut, n_steps, 0.0, hbar - dh, gxy.IMP_M1, env_policy)
    return (mp - mm) / (2.0 * dh)


def observables(beta, delta, n_max, d_cut, n_steps, hb=1e-3, hbar=0.01, dh=1e-3, env_policy=0):
    """All scalars of one (beta, Delta) point at zero field plus the field runs."""
    cv, l0 = specific_heat(beta, delta, n_max, d_cut, n_steps, hb, env_policy=env_policy)
    m = magnetisation(beta, delta, n_max, d_cut, n_steps, hbar, 0.0, gxy.IMP_M, env_policy)
    m1 = magnetisation(beta, delta, n_max, d_cut, n_steps, 0.0, hbar, gxy.IMP_M1, env_policy)
    chi = susceptibility(beta, delta, n_max, d_cut, n_steps, hbar, dh, "h", env_policy)
    chi1 = susceptibility(beta, delta, n_max, d_cut, n_steps, hbar, dh, "h1", env_policy)
    return Observables(lnz=l0, f=-l0 / beta, cv=cv, m=m, m1=m1, chi=chi, chi1=chi1)
