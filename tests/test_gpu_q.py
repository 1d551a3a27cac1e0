"""The q != 2 couplings (gxy_q) against the oracle: the FP64 form to 1e-10,
the block-sparse split form to 1e-9 (the charge rule is unchanged, so the
block structure is too)."""
import pytest

from oracle import hotrg as OH

from parity_points import Q_SHAPES

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


@pytest.mark.parametrize("beta,delta,nm,dcut,steps,q", Q_SHAPES)
def test_q_coupling_against_oracle(H, C, beta, delta, nm, dcut, steps, q):
    ref = OH.run_gxy(beta, delta, nm, dcut, steps, q=q).lnz_per_site
    fp = C.run([H.params(beta, delta, nm, dcut, steps, q=q)])[0]
    assert abs(fp.lnz_per_site - ref) <= 1e-10, fp.lnz_per_site - ref
    sp = C.run([H.params(beta, delta, nm, dcut, steps, prec=H.SPLIT_BF16, block_sparse=1, q=q)])[0]
    assert abs(sp.lnz_per_site - ref) <= 1e-9, sp.lnz_per_site - ref
    two = C.run([H.params(beta, delta, nm, dcut, steps)])[0]
    assert abs(two.lnz_per_site - fp.lnz_per_site) > 1e-6  # a different model from q = 2


def test_q_out_of_range_is_rejected(H, C):
    with pytest.raises(H.HotrgError) as e:
        C.run([H.params(1.0, 0.5, 2, 8, 4, q=5)])
    assert e.value.status == H.EINVAL
