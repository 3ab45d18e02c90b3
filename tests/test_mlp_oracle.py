"""Pins for the MLP cost-model oracle: finite differences, closed forms, Adam's definition."""
import numpy as np

from oracle import mlp


def flat_grad_check(params, X, y, n_probe, seed, h=1e-6):
    g = np.random.default_rng(seed)
    grads = mlp.backward(params, X, y)
    worst = 0.0
    for _ in range(n_probe):
        li = int(g.integers(len(params)))
        which = int(g.integers(2))
        arr = params[li][which]
        idx = tuple(int(g.integers(s)) for s in arr.shape)
        old = arr[idx]
        arr[idx] = old + h
        lp = mlp.loss(params, X, y)
        arr[idx] = old - h
        lm = mlp.loss(params, X, y)
        arr[idx] = old
        fd = (lp - lm) / (2 * h)
        an = grads[li][which][idx]
        worst = max(worst, abs(fd - an) / max(1e-8, abs(fd) + abs(an)))
    return worst


def test_gradients_match_central_differences_small():
    params = mlp.init(16, seed=1, hidden=(8, 8, 8))
    g = np.random.default_rng(2)
    X = g.standard_normal((32, 16))
    y = g.standard_normal(32)
    assert flat_grad_check(params, X, y, 300, seed=3) < 1e-6


def test_gradients_match_central_differences_full_size():
    params = mlp.init(16, seed=4)
    g = np.random.default_rng(5)
    X = g.standard_normal((64, 16))
    y = g.standard_normal(64)
    assert flat_grad_check(params, X, y, 200, seed=6) < 1e-5


def test_zero_weights_closed_form():
    params = [(np.zeros_like(W), np.zeros_like(b)) for W, b in mlp.init(16, seed=7)]
    W4, b4 = params[-1]
    params[-1] = (W4, np.array([0.75]))
    X = np.random.default_rng(8).standard_normal((10, 16))
    y = np.arange(10.0)
    p, _ = mlp.forward(params, X)
    assert np.all(p == 0.75)
    grads = mlp.backward(params, X, y)
    assert np.isclose(grads[-1][1][0], 2 * np.mean(0.75 - y))
    assert all(np.all(gW == 0) for gW, _ in grads[:-1])


def test_linear_region_is_matrix_product():
    # with nonnegative inputs and weights every unit is active: the net is affine
    g = np.random.default_rng(9)
    params = [(np.abs(W), np.abs(g.standard_normal(b.shape))) for W, b in mlp.init(16, seed=10)]
    X = np.abs(g.standard_normal((20, 16)))
    p, _ = mlp.forward(params, X)
    h = X
    for W, b in params:
        h = h @ W.T + b
    assert np.allclose(p, h[:, 0], rtol=1e-12, atol=0)


def test_adam_first_step_and_convergence():
    # first step moves each weight by lr * g / (|g| + eps) (bias corrections cancel)
    params = [(np.array([[1.0, -2.0]]), np.array([0.5]))]
    grads = [(np.array([[3.0, -1e-3]]), np.array([0.0]))]
    opt = mlp.Adam(params, lr=0.01)
    new = opt.step(params, grads)
    assert np.allclose(new[0][0], [[1.0 - 0.01 * 3 / (3 + 1e-8), -2.0 + 0.01 * 1e-3 / (1e-3 + 1e-8)]])
    assert new[0][1][0] == 0.5
    # minimise (w - 3)^2 from w = 0
    p = [(np.array([[0.0]]), np.array([0.0]))]
    opt = mlp.Adam(p, lr=0.05)
    for _ in range(2000):
        p = opt.step(p, [(2 * (p[0][0] - 3.0), np.array([0.0]))])
    assert abs(p[0][0][0, 0] - 3.0) < 1e-3
