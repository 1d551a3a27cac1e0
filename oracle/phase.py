"""Phase-boundary extraction from HOTRG observables (§3.4 results, Table 3.1).

TEST INFRASTRUCTURE (oracle): only tests/, the smoke check and the bench's
CPU legs use this module.

The thesis locates transitions from temperature scans:

* the peaks of the specific heat C_V(T) at zero field (the Ising line, and a
  BKT-side peak that overestimates T_BKT);
* the peak of the susceptibility chi(T) (Eq. 3.18, by a central difference
  of m in the field) at a small central field hbar: h with the M impurity for
  Delta > 0.36, h1 with the M1 impurity for Delta <= 0.36;
* the zero-field limit of the chi peak temperature, from a fit over several
  hbar.  The thesis gives the fit's parameters a, b, c for Delta = 0.32
  (a = 0.685, the T_c of Table 3.1 there) and cites the form to an earlier XY
  study; it is read here as T_p(hbar) = a + b hbar^c, so a = T_c(hbar -> 0).
  The form is a reading: parity of the fit against the thesis is unpinned;
  the least-squares solution itself is pinned (tests/test_oracle_phase.py).

Peaks are located on the sampled grid (a local maximum with a prominence
threshold) and refined by the vertex of the parabola through the maximum and
its two neighbours.  Every function here follows its definition directly.
"""

import math

import numpy as np
from scipy import optimize

from . import gxy
from .observables import magnetisation, lnz

C_LO, C_HI = 0.05, 2.0
C_GRID = 2001


# --- peaks -------------------------------------------------------------

def local_maxima(y):
    """Indices of the interior local maxima of y.

    A maximum is a run y[i] = ... = y[j] (i <= j, i >= 1, j <= n - 2) with
    y[i - 1] < y[i] and y[j] > y[j + 1]; it is reported at the middle
    (i + j) // 2 of the run.  End points are never maxima.
    """
    y = list(y)
    out = []
    i = 1
    while i < len(y) - 1:
        if y[i - 1] < y[i]:
            j = i
            while j + 1 < len(y) - 1 and y[j + 1] == y[i]:
                j += 1
            if y[j + 1] < y[j]:
                out.append((i + j) // 2)
            i = j + 1
        else:
            i += 1
    return out


def prominence(y, p):
    """Height of y[p] above the higher of its two bases.

    Walking left from p while the values stay <= y[p] (to the first strictly
    higher value or the end), the left base is the smallest value met; the
    right base likewise.  prominence = y[p] - max(left base, right base).
    """
    left = y[p]
    k = p
    while k >= 0 and y[k] <= y[p]:
        left = min(left, y[k])
        k -= 1
    right = y[p]
    k = p
    while k < len(y) and y[k] <= y[p]:
        right = min(right, y[k])
        k += 1
    return y[p] - max(left, right)


def vertex(x3, y3):
    """Vertex (x_v, y_v) of the parabola through three samples.

    The parabola y = A u^2 + B u + C in u = x - x3[1] interpolates the three
    points (the 3 x 3 Vandermonde system); x_v = x3[1] - B / (2 A),
    y_v = C - B^2 / (4 A).  Three equal values (the inside of a plateau of
    three or more samples) have no vertex: the middle sample is returned.
    """
    if y3[0] == y3[1] == y3[2]:
        return float(x3[1]), float(y3[1])
    u = np.asarray(x3, dtype=np.float64) - float(x3[1])
    V = np.stack([u * u, u, np.ones(3)], axis=1)
    A, B, C = np.linalg.solve(V, np.asarray(y3, dtype=np.float64))
    return float(x3[1]) - B / (2.0 * A), C - B * B / (4.0 * A)


def find_peaks(x, y, min_prominence=0.0, cap=None):
    """Refined peaks of y(x) on an ascending grid.

    Every interior local maximum with prominence >= min_prominence; with a
    cap, the cap most prominent (ties: smaller x first).  Returned in
    ascending x as a list of (x_v, y_v, prominence); (x_v, y_v) is the vertex
    of the parabola through the maximum and its two neighbours.
    """
    y = [float(v) for v in y]
    cands = [(p, prominence(y, p)) for p in local_maxima(y)]
    cands = [c for c in cands if c[1] >= min_prominence]
    if cap is not None:
        cands = sorted(cands, key=lambda c: (-c[1], c[0]))[:cap]
    cands.sort()
    out = []
    for p, pr in cands:
        xv, yv = vertex(x[p - 1:p + 2], y[p - 1:p + 2])
        out.append((xv, yv, pr))
    return out


# --- zero-field fit ------------------------------------------------------

def _ab(h, t, c):
    """(a, b, residuals) of the linear least squares t ~ a + b h^c at fixed c."""
    X = np.stack([np.ones_like(h), h ** c], axis=1)
    (a, b), *_ = np.linalg.lstsq(X, t, rcond=None)
    return a, b, t - a - b * h ** c


def _dprofile(h, t, c):
    """d RSS / dc of the profile RSS(c) = min over (a, b): by the envelope
    theorem only the explicit c dependence counts, -2 sum r_i b h_i^c ln h_i."""
    a, b, r = _ab(h, t, c)
    return -2.0 * float(np.sum(r * b * h ** c * np.log(h)))


def fit_tc(hbar, t_peak, c_lo=C_LO, c_hi=C_HI):
    """Least-squares fit T_p(hbar) = a + b hbar^c, c in [c_lo, c_hi].

    The profile RSS(c) (a, b solved linearly) is scanned on C_GRID points of
    [c_lo, c_hi] (c_lo = c_hi fixes c); around the best grid point the stationary point of the
    profile is found as a root of its derivative (brentq); a minimum on a
    bound stays there.  Errors are sqrt(diag(s^2 (J^T J)^-1)) with
    s^2 = RSS / (n - 3) and J the Jacobian of the model in (a, b, c) (zero when
    n = 3).  Returns a dict with a, b, c, their errors, rss, n, at_bound.
    """
    h = np.asarray(hbar, dtype=np.float64)
    t = np.asarray(t_peak, dtype=np.float64)
    n = len(h)
    if n < 3 or np.any(h <= 0) or not c_lo <= c_hi:
        raise ValueError("need >= 3 points with hbar > 0 and c_lo <= c_hi")
    grid = np.linspace(c_lo, c_hi, C_GRID)
    rss = [float(np.sum(_ab(h, t, c)[2] ** 2)) for c in grid]
    k = int(np.argmin(rss))
    at_bound = 0
    if c_lo == c_hi:  # c fixed: the linear fit alone
        c, at_bound = c_lo, 1
    elif k == 0 and _dprofile(h, t, grid[0]) >= 0:
        c, at_bound = grid[0], 1
    elif k == C_GRID - 1 and _dprofile(h, t, grid[-1]) <= 0:
        c, at_bound = grid[-1], 1
    else:
        lo, hi = grid[max(k - 1, 0)], grid[min(k + 1, C_GRID - 1)]
        c = optimize.brentq(lambda cc: _dprofile(h, t, cc), lo, hi, xtol=1e-15, rtol=4 * np.finfo(float).eps,
                            maxiter=500)
    a, b, r = _ab(h, t, c)
    s = float(np.sum(r * r))
    J = np.stack([np.ones_like(h), h ** c, b * h ** c * np.log(h)], axis=1)
    if n > 3:
        cov = s / (n - 3) * np.linalg.inv(J.T @ J)
        err = np.sqrt(np.diag(cov))
    else:
        err = np.zeros(3)
    return {"a": float(a), "b": float(b), "c": float(c), "a_err": float(err[0]), "b_err": float(err[1]),
            "c_err": float(err[2]), "rss": s, "n": n, "at_bound": at_bound}


# --- scans -----------------------------------------------------------------

FIELD_AUTO, FIELD_M, FIELD_M1 = "auto", gxy.IMP_M, gxy.IMP_M1


def field_for(delta, field=FIELD_AUTO):
    """The symmetry-breaking field of the chi scan: the thesis uses h (the M
    impurity) for Delta > 0.36 and h1 (the M1 impurity) for Delta <= 0.36."""
    if field == FIELD_AUTO:
        return FIELD_M if delta > 0.36 else FIELD_M1
    return field


def cv_scan(delta, n_max, d_cut, n_steps, temps, hb=1e-3, env_policy=0):
    """C_V(T) at h = h1 = 0 (Eq. 3.17 by the 3-point difference in beta = 1/T)."""
    out = []
    for T in temps:
        beta = 1.0 / T
        l0 = lnz(beta, delta, n_max, d_cut, n_steps, env_policy=env_policy)
        lp = lnz(beta + hb, delta, n_max, d_cut, n_steps, env_policy=env_policy)
        lm = lnz(beta - hb, delta, n_max, d_cut, n_steps, env_policy=env_policy)
        out.append(beta * beta * (lp - 2.0 * l0 + lm) / (hb * hb))
    return np.array(out)


def chi_scan(delta, n_max, d_cut, n_steps, temps, hbars, field=FIELD_AUTO, dh=1e-3, env_policy=0):
    """chi(T; hbar) = [m(hbar + dh) - m(hbar - dh)] / (2 dh), rows hbar, columns T."""
    kind = field_for(delta, field)
    out = np.zeros((len(hbars), len(temps)))
    for k, hb_ in enumerate(hbars):
        for j, T in enumerate(temps):
            beta = 1.0 / T
            if kind == FIELD_M:
                mp = magnetisation(beta, delta, n_max, d_cut, n_steps, hb_ + dh, 0.0, kind, env_policy)
                mm = magnetisation(beta, delta, n_max, d_cut, n_steps, hb_ - dh, 0.0, kind, env_policy)
            else:
                mp = magnetisation(beta, delta, n_max, d_cut, n_steps, 0.0, hb_ + dh, kind, env_policy)
                mm = magnetisation(beta, delta, n_max, d_cut, n_steps, 0.0, hb_ - dh, kind, env_policy)
            out[k, j] = (mp - mm) / (2.0 * dh)
    return out


def chi_peak(temps, chi_row, min_prominence=0.0):
    """Temperature of the most prominent chi peak of one row (nan if none)."""
    pk = find_peaks(temps, chi_row, min_prominence, cap=1)
    return pk[0][0] if pk else math.nan
