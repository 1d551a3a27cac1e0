"""Plain FP64 HOTRG (coarse-graining along one axis per step).

TEST INFRASTRUCTURE (oracle).  Restates §2.4.1 of the thesis step by step,
in the paper's order, with numpy library calls (einsum/tensordot for the
contractions, eigh for each symmetric eigenproblem) as the only primitives:

1. Fuse two tensors along the vertical axis (Eq. 2.11):
       M[(l1,l2),(r1,r2),u,d] = sum_i T[l1,r1,u,i] T[l2,r2,i,d]
   (T1 above T2; T1's down leg i meets T2's up leg).
2. HOSVD of M (Eq. 2.12).  The left unitary U of the mode-(l) matricisation is
   the eigenbasis of the environment E_L = M_(l) M_(l)^T; its eigenvalues are
   the squared norms |S_{i,:,:,:}|^2 of the core tensor.  E_L is formed
   without materialising M, by the exact regrouping
       A[(l1,i),(l1',j)] = sum_{r,u} T[l1,r,u,i] T[l1',r,u,j]
       B[(l2,i),(l2',j)] = sum_{r,d} T[l2,r,i,d] T[l2',r,j,d]
       E_L[(l1,l2),(l1',l2')] = sum_{i,j} A[l1,i,l1',j] B[l2,i,l2',j],
   and E_R likewise on the right legs.  (The test suite checks this against
   M_(l) M_(l)^T with M built explicitly.)
3. Truncation (§2.4.1, the eps_1 / eps_2 comparison and Eq. 2.15):
   eps_1 = discarded eigenvalue weight of E_L, eps_2 of E_R; the projector is
   the top-D' eigenvectors of E_L unless eps_2 < eps_1 (then of E_R).
   D' = min(D_cut, D_h^2).  Following the block-sparse remark of §2.3.1, each
   symmetry sector of E (fixed fused charge l1 + l2) is diagonalised on its
   own.  Reading of an unstated point: eigenvalues within tie_rtol * lambda_max
   (1e-9) of the D'-th largest form the cut cluster, filled by |q| ascending,
   then q descending, then lambda descending.  Charge conjugation makes the
   +q and -q blocks' eigenvalues exactly equal; 1e-9 keeps such pairs tied
   when the contractions carry ~1e-10 relative error (the split-precision
   form), so the kept member of a pair at the cut is fixed by the rule, not
   by rounding; eps_2 wins only if
   eps_2 < eps_1 * (1 - 1e-6), so ties keep the left side.  Mirror-image
   environments give eps_1 = eps_2 exactly; the 1e-6 margin keeps that tie
   from being decided by the rounding of the eigenvalue sums (about 1e-12
   relative), while a near-tie changes Z by far less than the truncation.
4. Coarse tensor (Eq. 2.16), contracted as s1 -> s2 -> s3:
       s1: W[x,l2,r1,u,i] = sum_{l1}    P[l1,l2,x] T[l1,r1,u,i]
       s2: Z[x,r1,u,r2,d] = sum_{l2,i}  W[x,l2,r1,u,i] T[l2,r2,i,d]
       s3: T'[x,x',u,d]   = sum_{r1,r2} Z[x,r1,u,r2,d] P[r1,r2,x']
5. Normalisation (§2.3.2 mentions normalising after each step; the scheme is
   unstated): c_k = ||T'||_F, T <- T' / c_k.  The next step coarse-grains
   the other axis (§2.4.1, after Eq. 2.16), done by relabelling
   (l, r, u, d) <- (u, d, l, r).
6. ln Z / N = ln c_0 + sum_k 2^-k ln c_k + 2^-n ln sum_{x,y} T[x,x,y,y]
   for N = 2^n sites on the periodic lattice (tTr of §2.4.1 closed on the
   final 1x1 network).

Impurity tensors (§3.4, Eq. 3.19-3.21; the update rule is cited there, not
stated): the impure tensor is coarse-grained with the pure tensor's projector
and norm, averaging its two positions in the fused pair:
    T_imp' = [P^T (T_imp above T) P + P^T (T above T_imp) P] / (2 c_k).
"""

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import gxy

TIE_RTOL = 1e-9
SIDE_RTOL = 1e-6
# The strict widths: exact ties only (the rounding level of an FP64 eigensolve)
# and a bare eps_2 < eps_1 comparison.  Every step records whether they would
# have kept the same side and the same eigenpairs, and how close each decision
# was to its threshold, so that the effect of the two widths above on a run can
# be read off without a second run.
STRICT_TIE_RTOL = 1e-12
STRICT_SIDE_RTOL = 0.0


@dataclass
class StepRecord:
    Dh: int
    Dv: int
    Dp: int
    eps_left: float
    eps_right: float  # nan when the right environment was not formed
    side: int  # 0 = left (U), 1 = right (V)
    ln_c: float
    kept: np.ndarray  # kept eigenvalues, in kept order
    # diagnostics of the two decisions of the step (no effect on the result):
    # strict_same: the strict widths keep the same side and the same (charge,
    # rank) eigenpairs; side_margin = eps_2 / eps_1 - 1 (nan without E_R);
    # cut_gap: smallest | |lam - lam_cut| - tie_rtol lam_max | / lam_max over the
    # chosen side's eigenvalues, the distance of the tie decision from its edge
    strict_same: bool = True
    side_margin: float = float("nan")
    cut_gap: float = float("inf")


@dataclass
class RunResult:
    lnz_per_site: float
    ln_c0: float
    ln_trace: float
    steps: List[StepRecord] = field(default_factory=list)
    imp_ratio: Optional[float] = None  # tTr(T_imp) / tTr(T) after the last step


def _einsum(spec, *ops):
    return np.einsum(spec, *ops, optimize=True)


def environment_left(T):
    """E_L as a (Dh^2, Dh^2) matrix, rows (l1, l2) with l1 major."""
    Dh = T.shape[0]
    A = _einsum("lrui,mruj->limj", T, T)
    B = _einsum("lrid,mrjd->limj", T, T)
    E = _einsum("aibj,cidj->acbd", A, B)
    return E.reshape(Dh * Dh, Dh * Dh)


def environment_right(T):
    """E_R as a (Dh^2, Dh^2) matrix, rows (r1, r2) with r1 major."""
    Dh = T.shape[1]
    A = _einsum("lrui,lsuj->risj", T, T)
    B = _einsum("lrid,lsjd->risj", T, T)
    E = _einsum("aibj,cidj->acbd", A, B)
    return E.reshape(Dh * Dh, Dh * Dh)


def fused_charges(qh, sym):
    q = (qh[:, None] + qh[None, :]).reshape(-1)
    if sym == "z2":
        q = np.mod(q, 2)
    elif sym == "none":
        q = np.zeros_like(q)
    return q


def sector_eigen(E, qf):
    """Eigenpairs of each charge sector of E: list of (lam, q, rank, vec)."""
    n = E.shape[0]
    cands = []
    for q in np.unique(qf):
        idx = np.nonzero(qf == q)[0]
        w, V = np.linalg.eigh(E[np.ix_(idx, idx)])
        order = np.argsort(-w, kind="stable")
        for rank, j in enumerate(order):
            v = np.zeros(n)
            v[idx] = V[:, j]
            cands.append((float(w[j]), int(q), rank, v))
    return cands


def select_kept(cands, Dp, tie_rtol=TIE_RTOL):
    """Indices (into cands) of the D' kept eigenpairs, in kept order."""
    lam = np.array([c[0] for c in cands])
    if len(cands) <= Dp:
        order = sorted(range(len(cands)), key=lambda a: (-lam[a], abs(cands[a][1]), -cands[a][1], cands[a][2]))
        return order
    lam_max = float(np.max(lam))
    tol = tie_rtol * abs(lam_max)
    by_lam = np.argsort(-lam, kind="stable")
    lam_cut = lam[by_lam[Dp - 1]]
    above = [a for a in range(len(cands)) if lam[a] > lam_cut + tol]
    above.sort(key=lambda a: (-lam[a], abs(cands[a][1]), -cands[a][1], cands[a][2]))
    cluster = [a for a in range(len(cands)) if abs(lam[a] - lam_cut) <= tol]
    cluster.sort(key=lambda a: (abs(cands[a][1]), -cands[a][1], -lam[a], cands[a][2]))
    need = Dp - len(above)
    return above + cluster[:need]


def _truncate(cands, keep):
    kept_set = set(keep)
    eps = math.fsum(cands[a][0] for a in range(len(cands)) if a not in kept_set)
    P = np.stack([cands[a][3] for a in keep], axis=1)
    qn = np.array([cands[a][1] for a in keep], dtype=np.int64)
    kept = np.array([cands[a][0] for a in keep])
    return P, qn, eps, kept


def truncation(E, qf, Dp, tie_rtol=TIE_RTOL):
    """(P, new charges, eps = discarded weight, kept eigenvalues) for one E."""
    cands = sector_eigen(E, qf)
    return _truncate(cands, select_kept(cands, Dp, tie_rtol))


def _labels(cands, keep):
    return sorted((cands[a][1], cands[a][2]) for a in keep)


def _cut_gap(cands, Dp, tie_rtol):
    """Distance of the nearest eigenvalue from the edge of the cut cluster, / lam_max."""
    if len(cands) <= Dp:
        return float("inf")
    lam = np.array([c[0] for c in cands])
    lam_max = float(np.max(np.abs(lam)))
    lam_cut = np.sort(lam)[::-1][Dp - 1]
    return float(np.min(np.abs(np.abs(lam - lam_cut) - tie_rtol * lam_max)) / lam_max)


def coarse(P3, T_up, T_dn):
    """Eq. 2.16 through s1 -> s2 -> s3, with T_up above T_dn."""
    W = _einsum("abx,arui->xbrui", P3, T_up)      # s1
    Z = _einsum("xbrui,bsid->xrusd", W, T_dn)     # s2 (the O(D^7) contraction)
    return _einsum("xrusd,rsy->xyud", Z, P3)      # s3


def hotrg_step(T, qh, qv, d_cut, sym="u1", env_policy=0, tie_rtol=TIE_RTOL, T_imp=None,
               side_rtol=SIDE_RTOL):
    """One coarse-graining step.

    T has shape (Dh, Dh, Dv, Dv) = [l, r, u, d]; qh / qv are the integer labels
    of the horizontal / vertical bond states.  Returns
    (T_next, qh_next, qv_next, record, T_imp_next) where the returned tensors
    are normalised by c_k and already relabelled for the next axis.
    """
    Dh, Dv = T.shape[0], T.shape[2]
    Dp = min(d_cut, Dh * Dh)
    qf = fused_charges(qh, sym)

    EL = environment_left(T)
    cands = sector_eigen(EL, qf)
    keep = select_kept(cands, Dp, tie_rtol)
    P, qn, eps_l, kept = _truncate(cands, keep)
    eps_r = float("nan")
    side = 0
    side_strict = 0
    chosen = (cands, keep)
    if env_policy == 0:
        ER = environment_right(T)
        candsR = sector_eigen(ER, qf)
        keepR = select_kept(candsR, Dp, tie_rtol)
        PR, qnR, eps_r, keptR = _truncate(candsR, keepR)
        if eps_r < eps_l * (1.0 - side_rtol):
            P, qn, kept, side = PR, qnR, keptR, 1
            chosen = (candsR, keepR)
        side_strict = 1 if eps_r < eps_l * (1.0 - STRICT_SIDE_RTOL) else 0
    cc, ck = chosen
    strict_same = side_strict == side and (
        _labels(cc, select_kept(cc, Dp, STRICT_TIE_RTOL)) == _labels(cc, ck))
    side_margin = eps_r / eps_l - 1.0 if (env_policy == 0 and eps_l != 0.0) else float("nan")

    P3 = P.reshape(Dh, Dh, Dp)
    Tn = coarse(P3, T, T)
    c = float(np.linalg.norm(Tn))
    Tn = Tn / c
    T_next = np.ascontiguousarray(Tn.transpose(2, 3, 0, 1))
    rec = StepRecord(Dh=Dh, Dv=Dv, Dp=Dp, eps_left=eps_l, eps_right=eps_r, side=side,
                     ln_c=math.log(c), kept=kept, strict_same=strict_same, side_margin=side_margin,
                     cut_gap=_cut_gap(cc, Dp, tie_rtol))
    imp_next = None
    if T_imp is not None:
        Ti = 0.5 * (coarse(P3, T_imp, T) + coarse(P3, T, T_imp)) / c
        imp_next = np.ascontiguousarray(Ti.transpose(2, 3, 0, 1))
    return T_next, qv.copy(), qn, rec, imp_next


def trace(T):
    """Closing trace of a 1x1 periodic network: sum_{x,y} T[x,x,y,y]."""
    return float(np.einsum("xxyy->", T))


def hotrg_run(T0, q0, n_steps, d_cut, sym="u1", env_policy=0, tie_rtol=TIE_RTOL,
              T_imp0=None, side_rtol=SIDE_RTOL, on_step=None) -> RunResult:
    """n_steps of HOTRG from site tensor T0 (all four legs labelled q0).

    Returns ln Z / N for N = 2^n_steps sites, per-step records, and (with an
    impurity tensor) the ratio tTr(T_imp)/tTr(T) of the final 1x1 network.
    """
    c0 = float(np.linalg.norm(T0))
    T = T0 / c0
    Ti = None if T_imp0 is None else T_imp0 / c0
    qh = np.asarray(q0, dtype=np.int64).copy()
    qv = qh.copy()
    steps = []
    acc = math.log(c0)
    for k in range(1, n_steps + 1):
        T, qh, qv, rec, Ti = hotrg_step(T, qh, qv, d_cut, sym, env_policy, tie_rtol, Ti, side_rtol)
        steps.append(rec)
        if on_step is not None:
            on_step(k, rec)
        acc += rec.ln_c * 2.0 ** (-k)
    tr = trace(T)
    if not tr > 0.0:
        raise FloatingPointError(f"non-positive closing trace {tr}")
    acc += math.log(tr) * 2.0 ** (-n_steps)
    res = RunResult(lnz_per_site=acc, ln_c0=math.log(c0), ln_trace=math.log(tr), steps=steps)
    if Ti is not None:
        res.imp_ratio = trace(Ti) / tr
    return res


def run_gxy(beta, delta, n_max, d_cut, n_steps, h=0.0, h1=0.0, env_policy=0,
            impurity=None, tie_rtol=TIE_RTOL, q=2, side_rtol=SIDE_RTOL, on_step=None) -> RunResult:
    """Convenience: build the gXY tensor (and an impurity) and run HOTRG."""
    sym = gxy.symmetry_of(h, h1)
    T0 = gxy.site_tensor(beta, delta, n_max, h, h1, gxy.PURE, q=q)
    Ti = None
    if impurity is not None:
        Ti = gxy.site_tensor(beta, delta, n_max, h, h1, impurity, q=q)
    q0 = gxy.leg_charges(n_max, sym)
    return hotrg_run(T0, q0, n_steps, d_cut, sym, env_policy, tie_rtol, Ti, side_rtol, on_step)
