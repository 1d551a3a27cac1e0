"""The tensor-core split-precision contraction engine (tcgen05, BF16 slices).

Exactness: operands whose values need only the leading slice give sums of
integers below 2^24, which the FP32 accumulator must return exactly; any
descriptor, swizzle or TMEM-layout mistake breaks bit equality.  Accuracy:
random FP64 operands against the FP64 definition of the product, normwise.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from gpu_util import to_dev, torch  # noqa: E402


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


def contract(H, C, prec, A, B):
    M, K = A.shape
    N = B.shape[0]
    dA, dB = to_dev(A), to_dev(B)
    dC = torch.full((M, N), float("nan"), dtype=torch.float64, device="cuda")
    H.hotrg_contract(C.handle, prec, M, N, K, dA.data_ptr(), K, dB.data_ptr(), K, dC.data_ptr(), N)
    torch.cuda.synchronize()
    return dC.cpu().numpy()


B1 = 7  # bits of the leading slice digit


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (256, 384, 4096), (300, 200, 100), (1, 1, 1), (130, 7, 4097),
                                   (64, 64, 9216)])
def test_leading_slice_is_exact(H, C, M, N, K):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    b1 = B1
    top = 2 ** b1 - 1
    a = rng.integers(-top, top + 1, size=(M, K))
    b = rng.integers(-top, top + 1, size=(N, K))
    a[:, 0] = top  # pin each row maximum to (2^b1 - 1) / 2^b1, so the row exponent is 0
    b[:, 0] = top
    A = a / 2.0 ** b1
    B = b / 2.0 ** b1
    ref = (a.astype(object) @ b.T.astype(object))  # exact integers
    ref = np.array(ref, dtype=np.float64) / 2.0 ** (2 * b1)
    got = contract(H, C, H.SPLIT_BF16, A, B)
    assert np.array_equal(got, ref), np.max(np.abs(got - ref))


def test_accumulation_beyond_one_chunk(H, C):
    # every leading product 127 * 127: 512 of them fill one exact chunk (< 2^24);
    # K = 8192 spans 16 chunks whose sum (2.6e8) is carried exactly across chunks
    for K in (512, 8192):
        A = np.full((128, K), 127 / 128.0)
        got = contract(H, C, H.SPLIT_BF16, A, A)
        assert np.all(got == K * (127 / 128.0) ** 2)
    # the second digit at its bound: diagonal-1 sums of 2 * 127 * 128 per k
    K = 1024
    A = np.full((128, K), 127 / 128.0 + 128 / 2.0 ** 15)
    got = contract(H, C, H.SPLIT_BF16, A, A)
    assert np.all(got == K * (127 / 128.0 + 128 / 2.0 ** 15) ** 2)


@pytest.mark.parametrize("M,N,K", [(512, 256, 4096), (257, 129, 81), (1000, 64, 576), (64, 640, 9216)])
def test_normwise_accuracy_random(H, C, M, N, K):
    rng = np.random.default_rng(K)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-12, 12, size=(M, 1)))
    B = rng.standard_normal((N, K)) * np.exp(rng.uniform(-12, 12, size=(N, 1)))
    ref = A @ B.T
    got = contract(H, C, H.SPLIT_BF16, A, B)
    bound = np.abs(A).max(1)[:, None] * np.abs(B).max(1)[None, :] * K
    rel = np.abs(got - ref) / bound
    assert rel.max() < 2.0 ** -29, rel.max()
    # FP32-class form: 3 slices (23 bits)
    got3 = contract(H, C, H.SPLIT_BF16_FAST, A, B)
    rel3 = np.abs(got3 - ref) / bound
    assert rel3.max() < 2.0 ** -21, rel3.max()


def test_positive_operands_have_no_drift(H, C):
    # all-positive data: a truncating accumulator would drift with K
    rng = np.random.default_rng(11)
    K = 4096
    A = np.abs(rng.standard_normal((256, K)))
    B = np.abs(rng.standard_normal((256, K)))
    ref = A @ B.T
    got = contract(H, C, H.SPLIT_BF16, A, B)
    rel = (got - ref) / ref
    assert np.abs(rel).max() < 2.0 ** -28 and abs(rel.mean()) < 2.0 ** -31


def test_fp64_engine_matches_definition(H, C):
    rng = np.random.default_rng(3)
    A = rng.standard_normal((70, 33))
    B = rng.standard_normal((45, 33))
    got = contract(H, C, H.FP64, A, B)
    assert np.allclose(got, A @ B.T, rtol=1e-14, atol=1e-13)


def test_contract_rejects_bad_arguments(H, C):
    d = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(H.HotrgError) as e:
        H.hotrg_contract(C.handle, H.SPLIT_BF16, 0, 4, 4, d.data_ptr(), 4, d.data_ptr(), 4, d.data_ptr(), 4)
    assert e.value.status == H.EINVAL
    with pytest.raises(H.HotrgError) as e:
        H.hotrg_contract(C.handle, H.SPLIT_BF16, 2, 2, 4, d.data_ptr(), 3, d.data_ptr(), 4, d.data_ptr(), 2)
    assert e.value.status == H.EINVAL
