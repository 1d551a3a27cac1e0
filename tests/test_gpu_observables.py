"""Observables (§3.4: f, C_V by Eq. 3.17, m and m1 from the impurity tensors of
Eq. 3.20 / 3.21, chi and chi1 by Eq. 3.18) at D_cut = 24 against the oracle.

Each point takes nine runs: ln Z at beta and beta +- hb; m at h = hbar +- dh
and hbar (the cos theta impurity, no conserved label: dense path); m1 at
h1 = hbar +- dh and hbar (the cos 2 theta impurity keeps the charge parity:
Z2 block form when block_sparse = 1).  The central differences amplify the
per-run error by beta^2 / hb^2 (C_V) and 1 / (2 dh) (chi), which sets the
tolerances below.
"""
import pytest

from oracle import observables as OO

pytestmark = pytest.mark.gpu

# well conditioned in every one of the nine runs (tests/test_oracle_conditioning.py); at
# (1.0, 0.5, 2, 24, 10) the h = 0.01 run is not: a 1e-15 input perturbation moves the oracle's
# own m by ~6e-7 (weakly broken U(1): nearly degenerate pairs straddle the cut)
POINTS = [(1.3, 0.7, 2, 24, 10)]
HB, HBAR, DH = 1e-3, 0.01, 1e-3


@pytest.fixture(scope="module")
def H():
    from paper_2609_20536_b300 import build
    build.build()
    from paper_2609_20536_b300 import hotrg
    return hotrg


@pytest.fixture(scope="module")
def C(H):
    c = H.Context()
    yield c
    c.close()


@pytest.fixture(scope="module")
def ref():
    return {p: OO.observables(*p, hb=HB, hbar=HBAR, dh=DH) for p in POINTS}


@pytest.mark.parametrize("point", POINTS)
# (the split form, the one scans use; the FP64 form's cos theta runs solve one 576-state block by
# FP64 Jacobi, minutes per point here, and its impurity path is covered at D_cut <= 16 by
# tests/test_gpu_fp64_parity.py and tests/test_gpu_block_sparse.py)
@pytest.mark.parametrize("prec_name,bs,tol", [("SPLIT_BF16", 1, 1e-9)])
def test_observables_dcut24(H, C, ref, point, prec_name, bs, tol):
    r = ref[point]
    o = C.observables([H.params(*point, prec=getattr(H, prec_name), block_sparse=bs)], hb=HB, hbar=HBAR, dh=DH)[0]
    assert o.status == 0
    beta = point[0]
    assert abs(o.lnz - r.lnz) <= tol
    assert abs(o.f - r.f) <= tol / beta
    assert abs(o.cv - r.cv) <= 4 * tol * beta * beta / HB ** 2, (o.cv, r.cv)
    assert abs(o.m - r.m) <= 10 * tol and abs(o.m1 - r.m1) <= 10 * tol, (o.m, r.m, o.m1, r.m1)
    assert abs(o.chi - r.chi) <= 10 * tol / DH and abs(o.chi1 - r.chi1) <= 10 * tol / DH, (o.chi, r.chi, o.chi1,
                                                                                          r.chi1)
    assert r.m > 0 and r.m1 > 0 and r.chi > 0 and r.chi1 > 0


def test_observables_batch_equals_single(H, C):
    pts = [H.params(*p, prec=H.SPLIT_BF16, block_sparse=1) for p in POINTS]
    one = [C.observables([p], hb=HB, hbar=HBAR, dh=DH)[0] for p in pts]
    many = C.observables_batch(pts, hb=HB, hbar=HBAR, dh=DH, nstreams=3)
    for a, b in zip(one, many):
        assert (a.lnz, a.cv, a.m, a.m1, a.chi, a.chi1) == (b.lnz, b.cv, b.m, b.m1, b.chi, b.chi1)
