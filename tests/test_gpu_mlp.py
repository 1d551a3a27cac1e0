"""Surrogate network kernels against the FP64 oracle MLP.

The GPU network uses BF16 weights with FP32 accumulation; the oracle runs in
FP64 on the same BF16-rounded weights, so the comparison isolates the FP32
accumulation and tanhf rounding."""
import numpy as np
import pytest

from oracle import mlp as OM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2609_20536_b300 import build
    build.build()
    from paper_2609_20536_b300 import hotrg
    return hotrg


def flatten(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def unflatten(flat):
    out, o = [], 0
    for a, b in zip(OM.SIZES[:-1], OM.SIZES[1:]):
        W = flat[o:o + a * b].reshape(a, b)
        o += a * b
        out.append((W, flat[o:o + b].copy()))
        o += b
    return out


def test_gradients_match_oracle(H):
    net = H.MLP(ensemble=2, seed=5)
    rng = np.random.default_rng(0)
    P = OM.init_params(11)
    P = [(W, rng.standard_normal(b.shape) * 0.1) for W, b in P]
    flat = flatten(P).astype(np.float32)
    net.set_params(1, flat)
    X = rng.uniform(-1.5, 1.5, size=(97, 2))
    T = rng.standard_normal((97, 4))
    loss, g = net.gradients(1, X, T)
    # oracle on the BF16-rounded weights the GPU holds (biases stay FP32)
    Pq = [(OM.weights_bf16(W.astype(np.float32)), b.astype(np.float32).astype(np.float64))
          for W, b in unflatten(flat.astype(np.float64))]
    Xq = X.astype(np.float32).astype(np.float64)
    Tq = T.astype(np.float32).astype(np.float64)
    ref_loss = OM.loss(Pq, Xq, Tq)
    ref = flatten(OM.backward(Pq, Xq, Tq))
    assert abs(loss - ref_loss) < 1e-5 * abs(ref_loss)
    scale = np.abs(ref).max()
    assert np.abs(g - ref).max() < 2e-5 * scale, np.abs(g - ref).max() / scale
    # the first member (different weights) gives different gradients
    _, g0 = net.gradients(0, X, T)
    assert np.abs(g0 - g).max() > 1e-3 * scale
    net.close()


def test_training_reduces_loss_and_is_deterministic(H):
    rng = np.random.default_rng(1)
    X = rng.uniform(-1, 1, size=(1024, 2))
    T = np.stack([np.sin(2 * X[:, 0]), np.cos(3 * X[:, 1]), X[:, 0] * X[:, 1], X[:, 0] ** 2 - 0.3], axis=1)
    a = H.MLP(ensemble=3, seed=7)
    l0 = np.mean((a.predict(X)[0] - T) ** 2)
    la = a.train(X, T, epochs=60, batch=128, lr=3e-3)
    l1 = np.mean((a.predict(X)[0] - T) ** 2)
    assert l1 < 0.05 * l0 and la < 0.05 * l0
    b = H.MLP(ensemble=3, seed=7)
    b.train(X, T, epochs=60, batch=128, lr=3e-3)
    assert np.array_equal(a.get_params(2), b.get_params(2))
    mean, spread = a.predict(X[:10])
    assert mean.shape == (10, 4) and np.all(spread > 0)
    a.close()
    b.close()
