"""Plain FP64 multilayer perceptron: the checker of the surrogate kernels.

TEST INFRASTRUCTURE (oracle).  The surrogate of the (beta, Delta) -> (f, C_V,
chi, chi1) map has no counterpart in the thesis; its specification is a
2 -> 128 -> 128 -> 128 -> 4 network with tanh hidden activations and a
linear output, trained by Adam on the mean squared error of standardised
targets.  This module writes that definition out:

  forward:   h_0 = x;  h_l = tanh(h_{l-1} W_l + b_l) for hidden layers;
             y = h_{L-1} W_L + b_L
  loss:      L = (1 / (n k)) sum_{i,j} (y_ij - t_ij)^2
  backward:  g_y = 2 (y - t) / (n k);  g_W = h^T g;  g_b = sum_rows g;
             g_h = g W^T;  through tanh: g_pre = g_h (1 - h^2)
  Adam:      m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
             w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)

Weights W_l are stored [in][out].  ``weights_bf16`` rounds a weight array to
bfloat16 (round to nearest even) so that the oracle can run on exactly the
values a BF16-weight network holds.  Pins: gradients against central finite
differences (tests/test_oracle_mlp.py).
"""

import numpy as np

SIZES = (2, 128, 128, 128, 4)


def init_params(seed, sizes=SIZES):
    """Glorot-uniform weights, zero biases (FP64)."""
    rng = np.random.default_rng(seed)
    params = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / (a + b))
        params.append((rng.uniform(-lim, lim, size=(a, b)), np.zeros(b)))
    return params


def weights_bf16(w):
    """Round FP64 values to the nearest bfloat16 (ties to even), returned as FP64."""
    f = np.asarray(w, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params, x):
    """Returns the output and the list of layer outputs (h_0 = x, ..., y)."""
    hs = [np.asarray(x, dtype=np.float64)]
    for li, (W, b) in enumerate(params):
        z = hs[-1] @ W + b
        hs.append(np.tanh(z) if li < len(params) - 1 else z)
    return hs[-1], hs


def loss(params, x, t):
    y, _ = forward(params, x)
    return float(np.mean((y - t) ** 2))


def backward(params, x, t):
    """Gradients of the MSE loss with respect to every (W, b)."""
    y, hs = forward(params, x)
    n, k = y.shape
    g = 2.0 * (y - t) / (n * k)
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        h = hs[li]
        grads[li] = (h.T @ g, g.sum(axis=0))
        if li > 0:
            g = (g @ W.T) * (1.0 - hs[li] ** 2)
    return grads


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.v = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        out = []
        for i, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
            new = []
            for j, (p, g) in enumerate(((W, gW), (b, gb))):
                m = self.b1 * self.m[i][j] + (1 - self.b1) * g
                v = self.b2 * self.v[i][j] + (1 - self.b2) * g * g
                mh = m / (1 - self.b1 ** self.t)
                vh = v / (1 - self.b2 ** self.t)
                new.append(p - self.lr * mh / (np.sqrt(vh) + self.eps))
                if j == 0:
                    mW, vW = m, v
                else:
                    mb, vb = m, v
            self.m[i] = (mW, mb)
            self.v[i] = (vW, vb)
            out.append(tuple(new))
        return out
