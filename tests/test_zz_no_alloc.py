"""The allocation-free contraction entry point (hotrg_contract_noalloc).

It serves callers that cannot allocate device memory (another allocator owns
the device budget, or cudaMalloc's implicit synchronisation is not
acceptable): its scratch is a static device array inside the library.  This
file is collected last so that a run stopping at its first failure has run
every other test already; it also passes alone in a fresh process.
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


# (form, bound on |error| / (max|a_row| max|b_row| K)): 5 slices carry 39 bits, 3 slices 23
FORMS = [("SPLIT_BF16", 2.0 ** -29), ("SPLIT_BF16_FAST", 2.0 ** -19)]


@pytest.mark.parametrize("form,tol", FORMS)
def test_noalloc_matches_contract_twice(H, form, tol):
    prec = getattr(H, form)
    rng = np.random.default_rng(2609)
    ctx = H.Context()
    for call, (M, N, K) in enumerate([(300, 200, 1000), (257, 129, 81)]):
        A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-6, 6, size=(M, 1)))
        B = rng.standard_normal((N, K)) * np.exp(rng.uniform(-6, 6, size=(N, 1)))
        dA, dB = to_dev(A), to_dev(B)
        ref = torch.full((M, N), float("nan"), dtype=torch.float64, device="cuda")
        got = torch.full((M, N), float("nan"), dtype=torch.float64, device="cuda")
        H.hotrg_contract(ctx.handle, prec, M, N, K, dA.data_ptr(), K, dB.data_ptr(), K, ref.data_ptr(), N)
        st = H.hotrg_contract_noalloc(prec, M, N, K, dA.data_ptr(), K, dB.data_ptr(), K, got.data_ptr(), N,
                                      torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert st == H.OK, (call, st)
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        bound = np.abs(A).max(1)[:, None] * np.abs(B).max(1)[None, :] * K
        assert np.all(np.isfinite(g))
        assert (np.abs(g - r) / bound).max() < tol
        assert (np.abs(g - A @ B.T) / bound).max() < tol
    ctx.close()


def test_noalloc_rejects_oversize(H):
    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    # 4096 x 4096 with K = 4096 needs 5 * 8192 * 4096 * 2 bytes of slices: above the 32 MiB scratch
    st = H.hotrg_contract_noalloc(H.SPLIT_BF16, 4096, 4096, 4096, d.data_ptr(), 4096, d.data_ptr(), 4096,
                                  d.data_ptr(), 4096, 0)
    assert st == H.EINVAL
