"""Pins of the oracle's eps_1 / eps_2 rule (§2.4.1, the comparison after Eq. 2.12)
and of what the two widths of its reading (the side margin and the cut-cluster
width) change.

The rule: eps_1 and eps_2 are the weights the truncation discards from the
left and right matricisations of the fused tensor M (Eq. 2.11); the projector
comes from the side that discards less.  The pins use tensors without mirror
symmetry, so that eps_1 != eps_2 by a wide margin, and rebuild everything
from M itself (not from the oracle's regrouped environments):
  * eps_1, eps_2 are the sums of the discarded eigenvalues of M_(l) M_(l)^T and
    M_(r) M_(r)^T (M formed explicitly, numpy's eigvalsh);
  * by Eckart-Young the chosen side's truncation error ||M - P P^T M||^2 on its
    mode equals min(eps_1, eps_2);
  * c_k of the coarse tensor P^T M P (Eq. 2.16) built with the smaller-eps
    side's P equals the oracle's, and differs from the other side's;
  * mirroring the tensor (l <-> r, with the horizontal labels negated so the
    charge rule still holds) swaps eps_1 and eps_2 and flips the side.
Planted mistakes (the comparison inverted; always the left side) must fail
these pins.
"""
import inspect

import numpy as np
import pytest

from oracle import hotrg as OH

from parity_points import BATCH, FP64_SHAPES, SPLIT_SHAPES


def random_charged(seed, Dh=5, Dv=4):
    rng = np.random.default_rng(seed)
    qh = rng.integers(-2, 3, size=Dh)
    qv = rng.integers(-1, 2, size=Dv)
    T = rng.standard_normal((Dh, Dh, Dv, Dv))
    mask = (qh[:, None, None, None] + qv[None, None, :, None]) == (qh[None, :, None, None] + qv[None, None, None, :])
    T = T * mask
    return T / np.linalg.norm(T), qh, qv


def fused(T):
    """M[(l1,l2),(r1,r2),u,d] = sum_i T[l1,r1,u,i] T[l2,r2,i,d] (Eq. 2.11), as an explicit array."""
    Dh, Dv = T.shape[0], T.shape[2]
    M = np.zeros((Dh, Dh, Dh, Dh, Dv, Dv))
    for l1 in range(Dh):
        for l2 in range(Dh):
            # sum over the shared vertical bond i
            M[l1, l2] = np.einsum("rui,sid->rsud", T[l1], T[l2])
    return M  # [l1, l2, r1, r2, u, d]


def top_projector(Mmat, Dp):
    w, V = np.linalg.eigh(Mmat @ Mmat.T)
    order = np.argsort(-w)
    return V[:, order[:Dp]], float(np.sum(w[order[Dp:]]))


def side_rule_failures(step, seeds=(0, 1, 2), d_cut=8):
    """Everything the pins check, for a step function with the oracle's signature."""
    bad = []
    for seed in seeds:
        T, qh, qv = random_charged(seed)
        Dh, Dv = T.shape[0], T.shape[2]
        Dp = min(d_cut, Dh * Dh)
        _, _, _, rec, _ = step(T, qh, qv, d_cut, "u1")
        M = fused(T)
        ML = M.reshape(Dh * Dh, -1)                                   # mode (l1, l2)
        MR = M.transpose(2, 3, 0, 1, 4, 5).reshape(Dh * Dh, -1)       # mode (r1, r2)
        PL, e1 = top_projector(ML, Dp)
        PR, e2 = top_projector(MR, Dp)
        if abs(e1 - e2) < 1e-3 * max(e1, e2):
            bad.append((seed, "tensor too symmetric for the pin"))
            continue
        if not abs(rec.eps_left - e1) <= 1e-12 * np.trace(ML @ ML.T):
            bad.append((seed, "eps_1", rec.eps_left, e1))
        if not abs(rec.eps_right - e2) <= 1e-12 * np.trace(MR @ MR.T):
            bad.append((seed, "eps_2", rec.eps_right, e2))
        want = 0 if e1 <= e2 else 1
        if rec.side != want:
            bad.append((seed, "side", rec.side, want))
        # Eckart-Young: the kept side's mode truncation error is the smaller eps
        P, Mm = (PL, ML) if want == 0 else (PR, MR)
        err = float(np.linalg.norm(Mm - P @ (P.T @ Mm)) ** 2)
        if not abs(err - min(e1, e2)) <= 1e-10 * max(e1, e2):
            bad.append((seed, "truncation error", err, min(e1, e2)))
        # c_k of P^T M P with the kept side's projector (gauge invariant), and not with the other's
        def ln_c(P3):
            Tc = np.einsum("abx,abcduv,cdy->xyuv", P3, M, P3)
            return float(np.log(np.linalg.norm(Tc)))
        lc_want = ln_c((PL if want == 0 else PR).reshape(Dh, Dh, Dp))
        lc_other = ln_c((PR if want == 0 else PL).reshape(Dh, Dh, Dp))
        if not abs(rec.ln_c - lc_want) <= 1e-12:
            bad.append((seed, "ln c_k", rec.ln_c, lc_want))
        if not abs(lc_want - lc_other) > 1e-8:
            bad.append((seed, "the two sides give the same c_k: pin not discriminating"))
        # mirror image: l <-> r with negated horizontal labels keeps the charge rule
        Tm = np.ascontiguousarray(T.transpose(1, 0, 2, 3))
        _, _, _, rm, _ = step(Tm, -qh, qv, d_cut, "u1")
        if not (abs(rm.eps_left - rec.eps_right) <= 1e-12 * abs(rec.eps_right) + 1e-15 and
                abs(rm.eps_right - rec.eps_left) <= 1e-12 * abs(rec.eps_left) + 1e-15):
            bad.append((seed, "mirror swaps eps", rm.eps_left, rm.eps_right))
        if rm.side != 1 - rec.side:
            bad.append((seed, "mirror flips the side", rm.side, rec.side))
        if not abs(rm.ln_c - rec.ln_c) <= 1e-12:
            bad.append((seed, "mirror keeps c_k", rm.ln_c, rec.ln_c))
    return bad


def test_fused_tensor_is_eq_2_11():
    # spot check of the explicit M against the definition, element by element
    T, _, _ = random_charged(5, Dh=3, Dv=2)
    M = fused(T)
    for (l1, l2, r1, r2, u, d) in [(0, 1, 2, 0, 1, 0), (2, 2, 1, 0, 0, 1), (1, 0, 1, 1, 1, 1)]:
        want = sum(T[l1, r1, u, i] * T[l2, r2, i, d] for i in range(2))
        assert abs(M[l1, l2, r1, r2, u, d] - want) <= 1e-15


def test_side_rule_pins_hold_for_the_oracle():
    assert side_rule_failures(OH.hotrg_step) == []


def _mutant(old, new):
    """OH.hotrg_step with one planted change, compiled in the oracle module's namespace (CPU only)."""
    src = inspect.getsource(OH.hotrg_step)
    assert old in src
    ns = dict(vars(OH))
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    return ns["hotrg_step"]


@pytest.mark.parametrize("old,new", [
    ("if eps_r < eps_l * (1.0 - side_rtol):", "if eps_r > eps_l * (1.0 - side_rtol):"),   # comparison inverted
    ("if eps_r < eps_l * (1.0 - side_rtol):", "if False:"),                                # always the left side
    ("if eps_r < eps_l * (1.0 - side_rtol):", "if True:"),                                 # always the right side
])
def test_planted_side_rule_mistakes_fail_the_pins(old, new):
    assert side_rule_failures(_mutant(old, new)) != []


# The widths of the reading, on the GPU parity points: a strict rerun (cluster width
# 1e-12, bare eps comparison) must give the same ln Z / N to rounding, and every step
# where the strict widths decide otherwise must be an exact mirror tie
# (|eps_2 / eps_1 - 1| at rounding level), where either side gives the same Z.
STRICT_POINTS = [p for p in FP64_SHAPES + SPLIT_SHAPES[:2] + SPLIT_SHAPES[3:4] + BATCH[:4] if p[3] <= 16]


@pytest.mark.parametrize("point", STRICT_POINTS)
def test_strict_widths_change_nothing_on_parity_points(point):
    a = OH.run_gxy(*point)
    b = OH.run_gxy(*point, tie_rtol=OH.STRICT_TIE_RTOL, side_rtol=OH.STRICT_SIDE_RTOL)
    assert abs(a.lnz_per_site - b.lnz_per_site) <= 1e-13
    for k, r in enumerate(a.steps):
        if not r.strict_same:
            assert abs(r.side_margin) <= 1e-12, (k + 1, r.side_margin)


def test_strict_widths_at_dcut64_move_lnz_below_1e12():
    # The first D_cut = 64 workload point, stored by the oracle with the reading's widths and with
    # the strict ones (tests/golden/make_oracle_goldens.py headline0 and headline0_strict).  There
    # the 1e-6 side margin decides genuine near-ties -- steps where eps_2 < eps_1 by up to 6e-7
    # relative keep the left side -- so the two runs take different sides from step 5 on; each
    # decision sits inside the margin (both sides truncate the same weight to 6 digits), single
    # ln c_k move by ~1e-9, ln Z / N by 7e-13.
    import json
    import os
    gold = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    g = json.load(open(os.path.join(gold, "oracle_headline0.json")))
    s = json.load(open(os.path.join(gold, "strict_headline0.json")))
    assert (g["tie_rtol"], g["side_rtol"]) == (OH.TIE_RTOL, OH.SIDE_RTOL)
    assert s["strict"] and (s["tie_rtol"], s["side_rtol"]) == (OH.STRICT_TIE_RTOL, OH.STRICT_SIDE_RTOL)
    assert abs(g["lnz_per_site"] - s["lnz_per_site"]) <= 1e-12
    differing = [st for st in g["steps"] if not st["strict_same"]]
    assert differing  # the widths do decide here
    for st in differing:
        assert abs(st["side_margin"]) < OH.SIDE_RTOL, (st["k"], st["side_margin"])
