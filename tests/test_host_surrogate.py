"""Host-only parts of the surrogate driver (no device work): the input and
output standardisation is the column mean and population standard deviation,
with a constant column mapped to a unit scale."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def H():
    from paper_2609_20536_b300 import build
    build.build()
    from paper_2609_20536_b300 import hotrg
    return hotrg


def test_scaling_is_mean_and_population_std(H):
    rng = np.random.default_rng(3)
    X = np.column_stack([rng.uniform(0.5, 2.0, 300), rng.uniform(0.0, 1.0, 300)])
    Y = rng.normal(size=(300, 4)) * [0.1, 5.0, 30.0, 1.0] + [-1.0, 2.0, 0.0, 7.0]
    Y[:, 3] = 7.0  # constant column
    s = H.hotrg_scaling_fit(X, Y)
    np.testing.assert_allclose(s.x_mean[:], X.mean(0), rtol=1e-13)
    np.testing.assert_allclose(s.x_std[:], X.std(0), rtol=1e-12)
    np.testing.assert_allclose(s.y_mean[:], Y.mean(0), rtol=1e-13)
    np.testing.assert_allclose(s.y_std[:3], Y[:, :3].std(0), rtol=1e-12)
    assert s.y_std[3] == 1.0
    # standardised columns then have mean 0 and unit variance
    Z = (Y[:, :3] - np.array(s.y_mean[:3])) / np.array(s.y_std[:3])
    np.testing.assert_allclose(Z.mean(0), 0.0, atol=1e-13)
    np.testing.assert_allclose(Z.var(0), 1.0, rtol=1e-12)


def test_scaling_rejects_empty_and_nonfinite(H):
    with pytest.raises(H.HotrgError):
        H.hotrg_scaling_fit(np.zeros((0, 2)), np.zeros((0, 4)))
    X = np.ones((4, 2))
    Y = np.ones((4, 4))
    Y[2, 1] = np.nan
    with pytest.raises(H.HotrgError):
        H.hotrg_scaling_fit(X, Y)
