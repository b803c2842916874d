"""Pins of the numpy MLP reference: central finite differences of the loss, closed
forms (zero weights give the bias; ReLU cuts negative pre-activations) and the
packed layout's size."""
import numpy as np

from oracle import mlp


def _data(n, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, mlp.IN))
    y = rng.normal(size=(n, mlp.OUT))
    mask = (rng.random((n, mlp.OUT)) < 0.8).astype(np.float64)
    return x, y, mask


def test_param_count_matches_layout():
    assert mlp.PARAMS == 16 * 64 + 64 + 64 * 64 + 64 + 64 * 10 + 10 == 5898


def test_gradient_matches_central_finite_differences():
    x, y, m = _data(7)
    theta = mlp.init(3)
    inv = 1.0 / m.sum()
    _, g = mlp.loss_grad(theta, x, y, m, inv)
    rng = np.random.default_rng(1)
    idx = rng.choice(mlp.PARAMS, 60, replace=False)
    for name, (lo, hi) in {"W1": (0, 1024), "b3": (5888, 5898)}.items():
        idx = np.concatenate([idx, [lo, hi - 1]])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        num = (mlp.loss(tp, x, y, m, inv) - mlp.loss(tm, x, y, m, inv)) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 + 1e-5 * abs(num), (i, num, g[i])


def test_zero_weights_output_the_bias_and_relu_cuts():
    p = mlp.unpack(np.zeros(mlp.PARAMS))
    p = {k: v.copy() for k, v in p.items()}
    p["b3"][:] = np.arange(10)
    yh, _ = mlp.forward(mlp.pack(p), np.ones((3, 16)))
    np.testing.assert_array_equal(yh, np.tile(np.arange(10.0), (3, 1)))
    p["b1"][:] = -1.0  # every hidden unit of layer 1 negative -> h1 = 0
    p["W2"][:] = 5.0
    p["b2"][:] = 0.0
    p["W3"][:] = 1.0
    yh, (x, a1, h1, a2, h2) = mlp.forward(mlp.pack(p), np.zeros((2, 16)))
    assert (h1 == 0).all() and (h2 == 0).all()
    np.testing.assert_array_equal(yh, np.tile(np.arange(10.0), (2, 1)))


def test_masked_targets_do_not_contribute():
    x, y, m = _data(5, seed=4)
    theta = mlp.init(5)
    y2 = y.copy()
    y2[m == 0] += 1000.0
    L1, g1 = mlp.loss_grad(theta, x, y, m, 0.1)
    L2, g2 = mlp.loss_grad(theta, x, y2, m, 0.1)
    assert L1 == L2
    np.testing.assert_array_equal(g1, g2)
