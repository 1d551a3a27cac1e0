"""Conditioning of the GPU parity points, checked on the oracle alone.

A parity tolerance is only meaningful where the quantity is fixed to that
tolerance by the arithmetic: if a relative perturbation eta of the input
tensor (the size of one rounding of the form under test) moves ln Z / N by
more than the tolerance, two correct programs may disagree by that much.
Each point is run with the input multiplied by (1 + eta * N(0,1)) for two
seeds; the largest move must stay at least five times below the tolerance.
"""
import numpy as np
import pytest

from oracle import gxy
from oracle import hotrg as OH

from parity_points import BATCH_ORACLE, DRIFT_SHAPES, FP64_SHAPES, ILL_CONDITIONED, SPLIT_SHAPES


def spread(point, eta, seeds=(1, 2)):
    beta, delta, nm, dcut, steps = point
    T0 = gxy.site_tensor(beta, delta, nm)
    q0 = gxy.leg_charges(nm, "u1")
    ref = OH.hotrg_run(T0, q0, steps, dcut, "u1").lnz_per_site
    worst = 0.0
    for s in seeds:
        rng = np.random.default_rng(s)
        Tp = T0 * (1.0 + eta * rng.standard_normal(T0.shape))
        worst = max(worst, abs(OH.hotrg_run(Tp, q0, steps, dcut, "u1").lnz_per_site - ref))
    return worst


@pytest.mark.parametrize("point", FP64_SHAPES)
def test_fp64_points_are_well_conditioned(point):
    assert spread(point, 1e-15) <= 2e-12


@pytest.mark.parametrize("point", SPLIT_SHAPES + BATCH_ORACLE + DRIFT_SHAPES)
def test_split_points_are_well_conditioned(point):
    # the split form's per-step ln c_k are accurate to ~1e-10 relative
    assert spread(point, 1e-10) <= 2e-10


def test_ill_conditioned_counter_example():
    # the same model and cut, four steps further: rounding-level noise is
    # amplified past any FP64 parity tolerance
    assert spread(ILL_CONDITIONED, 1e-15) > 1e-9
    short = ILL_CONDITIONED[:4] + (10,)
    assert spread(short, 1e-15) <= 2e-12
    assert spread(short, 1e-10) > 1e-9


def label_sum_bound(point):
    """Largest |q_x| + |q_h| + |q_v| over the steps of the oracle's run: a bound on the
    signed three-leg label sums of the block-sparse products (new bond, horizontal, vertical)."""
    beta, delta, nm, dcut, steps = point
    T = gxy.site_tensor(beta, delta, nm)
    T = T / np.linalg.norm(T)
    qh = np.asarray(gxy.leg_charges(nm, "u1"), dtype=np.int64)
    qv = qh.copy()
    worst = 0
    for _ in range(steps):
        qh0, qv0 = qh, qv
        T, qh, qv, _, _ = OH.hotrg_step(T, qh, qv, dcut, "u1", 0, OH.TIE_RTOL, None)
        worst = max(worst, int(np.abs(qv).max() + np.abs(qh0).max() + np.abs(qv0).max()))
    return worst, int(np.ptp(qh)), int(np.ptp(qv))


@pytest.mark.parametrize("point", DRIFT_SHAPES)
def test_drift_points_leave_the_centred_label_range(point):
    # the kept window really drifts (label sums beyond 64), while its width stays small
    worst, wh, wv = label_sum_bound(point)
    assert worst > 64 and wh < 40 and wv < 40


# The observables test points (tests/test_gpu_observables.py): the cos theta impurity run at
# h = hbar = 0.01 has no conserved label, and at small h nearly degenerate pairs can straddle
# the cut -- there rounding-level noise decides the kept state.  The chosen points are
# conditioned to 1e-15; the first one below is the counter-example.
def m_spread(point, h, eta=1e-15, seeds=(1, 2)):
    beta, delta, nm, dcut, steps = point
    T0 = gxy.site_tensor(beta, delta, nm, h, 0.0, gxy.PURE)
    Ti = gxy.site_tensor(beta, delta, nm, h, 0.0, gxy.IMP_M)
    q0 = gxy.leg_charges(nm, "none")
    ref = OH.hotrg_run(T0, q0, steps, dcut, "none", T_imp0=Ti).imp_ratio
    worst = 0.0
    for s in seeds:
        rng = np.random.default_rng(s)
        Tp = T0 * (1.0 + eta * rng.standard_normal(T0.shape))
        worst = max(worst, abs(OH.hotrg_run(Tp, q0, steps, dcut, "none", T_imp0=Ti).imp_ratio - ref))
    return worst


@pytest.mark.parametrize("point", [(1.3, 0.7, 2, 24, 10), (0.7, 0.9, 2, 24, 10)])
def test_observables_points_are_well_conditioned(point):
    assert m_spread(point, 0.01) <= 1e-12


def test_observables_counter_example_is_ill_conditioned():
    assert m_spread((1.0, 0.5, 2, 24, 10), 0.01) > 1e-8
