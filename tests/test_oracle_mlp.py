"""Pins of the oracle MLP: gradients against central finite differences, the
Adam update against its closed form on a quadratic, bf16 rounding."""
import numpy as np

from oracle import mlp


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    sizes = (2, 7, 5, 3)
    P = mlp.init_params(3, sizes)
    P = [(W, rng.standard_normal(b.shape) * 0.1) for W, b in P]
    x = rng.standard_normal((9, 2))
    t = rng.standard_normal((9, 3))
    G = mlp.backward(P, x, t)
    eps = 1e-6
    for li, (W, b) in enumerate(P):
        for arr_i, arr in enumerate((W, b)):
            num = np.zeros_like(arr)
            for idx in np.ndindex(arr.shape):
                old = arr[idx]
                arr[idx] = old + eps
                lp = mlp.loss(P, x, t)
                arr[idx] = old - eps
                lm = mlp.loss(P, x, t)
                arr[idx] = old
                num[idx] = (lp - lm) / (2 * eps)
            assert np.allclose(G[li][arr_i], num, rtol=1e-6, atol=1e-9)


def test_adam_first_step_is_signed_lr():
    # after one step from zero moments, Adam moves every weight by -lr * sign(g)
    P = [(np.array([[1.0, -2.0]]), np.array([0.5, 0.0]))]
    G = [(np.array([[3.0, -1e-3]]), np.array([-4.0, 2.0]))]
    opt = mlp.Adam(P, lr=0.01)
    new = opt.step(P, G)
    assert np.allclose(new[0][0], [[1.0 - 0.01, -2.0 + 0.01]], atol=1e-7)
    assert np.allclose(new[0][1], [0.5 + 0.01, 0.0 - 0.01], atol=1e-7)


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, -3.14159265])
    r = mlp.weights_bf16(v)
    assert r[0] == 1.0
    assert r[1] == 1.0  # exactly halfway: ties to even
    assert r[2] == 1.0  # below halfway
    assert r[3] == 1.0 + 2 ** -7
    assert abs(r[4] + 3.140625) < 1e-12
