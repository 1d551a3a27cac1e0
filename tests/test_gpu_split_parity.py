"""End-to-end parity of the split-precision forms against the FP64 oracle.

HOTRG_SPLIT_BF16 must reach |d lnZ/N| <= 1e-9 (the target of the split
form); HOTRG_SPLIT_BF16_FAST is the FP32 accuracy class and only has to stay
within 1e-6 (its measured error is reported by the bench)."""
import pytest

from oracle import gxy
from oracle import hotrg as OH

from parity_points import SPLIT_SHAPES

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("beta,delta,nm,dcut,steps", SPLIT_SHAPES)
def test_split_bf16_lnz(H, C, beta, delta, nm, dcut, steps):
    ref = OH.run_gxy(beta, delta, nm, dcut, steps)
    res = C.run([H.params(beta, delta, nm, dcut, steps, prec=H.SPLIT_BF16)])[0]
    assert res.status == 0
    assert abs(res.lnz_per_site - ref.lnz_per_site) <= 1e-9, res.lnz_per_site - ref.lnz_per_site
    for k, rs in enumerate(ref.steps):
        assert res.step[k].dprime == rs.Dp
        assert abs(res.step[k].ln_c - rs.ln_c) <= 1e-7 * max(1.0, abs(rs.ln_c))


def test_split_fast_lnz(H, C):
    ref = OH.run_gxy(1.0, 0.5, 2, 16, 20)
    res = C.run([H.params(1.0, 0.5, 2, 16, 20, prec=H.SPLIT_BF16_FAST)])[0]
    assert res.status == 0
    assert abs(res.lnz_per_site - ref.lnz_per_site) <= 1e-6


def test_split_impurity(H, C):
    ref = OH.run_gxy(1.1, 0.4, 2, 10, 10, h1=0.03, impurity=gxy.IMP_M1)
    res = C.run([H.params(1.1, 0.4, 2, 10, 10, h1=0.03, prec=H.SPLIT_BF16)], imp_kind=H.T_IMP_M1)[0]
    assert abs(res.lnz_per_site - ref.lnz_per_site) <= 1e-9
    assert abs(res.imp_ratio - ref.imp_ratio) <= 1e-8


def test_split_ising(H, C):
    ref = OH.hotrg_run(gxy.ising_tensor(0.6), gxy.ising_charges(), 30, 16, "z2")
    res = C.run([H.params(0.6, 0.0, 0, 16, 30, tkind=H.T_ISING, prec=H.SPLIT_BF16)])[0]
    assert abs(res.lnz_per_site - ref.lnz_per_site) <= 1e-9
