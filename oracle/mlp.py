"""Learned cost model oracle -- TEST INFRASTRUCTURE ONLY.

A plain numpy FP64 restatement of the MLP the tuner trains on the GPU: input
features -> 3 hidden layers of 128 ReLU units -> one linear output, the
predicted log runtime; loss = mean squared error; optimiser = Adam
(Kingma & Ba 2015, Algorithm 1: m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
m^ = m / (1 - b1^t), v^ = v / (1 - b2^t), w <- w - lr m^ / (sqrt(v^) + eps)).

Layer l computes z_l = h_{l-1} W_l^T + b_l (W_l: out x in, row-major) and
h_l = relu(z_l) for the hidden layers.  Backward is the textbook chain rule.
Parity is pinned by central finite differences and closed-form cases in
tests/test_mlp_oracle.py.
"""
from __future__ import annotations

import numpy as np

HIDDEN = (128, 128, 128)


def init(n_in, seed, hidden=HIDDEN):
    """He-uniform weights, zero biases (same recipe the GPU side is given as input)."""
    g = np.random.default_rng(seed)
    dims = (n_in,) + tuple(hidden) + (1,)
    params = []
    for i in range(len(dims) - 1):
        lim = np.sqrt(6.0 / dims[i])
        params.append((g.uniform(-lim, lim, size=(dims[i + 1], dims[i])), np.zeros(dims[i + 1])))
    return params


def forward(params, X):
    """Returns (prediction (batch,), cache of layer inputs/pre-activations)."""
    h = np.asarray(X, dtype=np.float64)
    cache = []
    for li, (W, b) in enumerate(params):
        z = h @ W.T + b
        cache.append((h, z))
        h = np.maximum(z, 0.0) if li < len(params) - 1 else z
    return h[:, 0], cache


def loss(params, X, y):
    p, _ = forward(params, X)
    return float(np.mean((p - y) ** 2))


def backward(params, X, y):
    """Gradients of the MSE loss w.r.t. every (W, b)."""
    p, cache = forward(params, X)
    B = X.shape[0]
    g = (2.0 / B) * (p - y)[:, None]  # dL/dz of the output layer
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        h, z = cache[li]
        if li < len(params) - 1:
            g = g * (z > 0)
        W, _ = params[li]
        grads[li] = (g.T @ h, g.sum(axis=0))
        g = g @ W
    return grads


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.t = 0
        self.m = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.v = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]

    def step(self, params, grads):
        self.t += 1
        out = []
        for i, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
            new = []
            for j, (w, g) in enumerate(((W, gW), (b, gb))):
                m = self.b1 * self.m[i][j] + (1 - self.b1) * g
                v = self.b2 * self.v[i][j] + (1 - self.b2) * g * g
                mh = m / (1 - self.b1 ** self.t)
                vh = v / (1 - self.b2 ** self.t)
                new.append(w - self.lr * mh / (np.sqrt(vh) + self.eps))
                if j == 0:
                    mW, vW = m, v
                else:
                    self.m[i] = (mW, m)
                    self.v[i] = (vW, v)
            out.append((new[0], new[1]))
        return out
