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


def test_adam_two_steps_worked_by_hand():
    # Kingma & Ba (2015), Algorithm 1, with beta1 = 9/10, beta2 = 999/1000, lr = 1/10,
    # one parameter starting at 1 with gradients 1/2 and then -1/4.
    #   t = 1: m = (1/10)(1/2) = 1/20, v = (1/1000)(1/4) = 1/4000,
    #          m_hat = (1/20)/(1/10) = 1/2, v_hat = (1/4000)/(1/1000) = 1/4,
    #          theta = 1 - (1/10)(1/2)/(1/2 + eps)            (a step of lr * sign(g))
    #   t = 2: m = (9/10)(1/20) - (1/10)(1/4) = 1/50,
    #          v = (999/1000)(1/4000) + (1/1000)(1/16) = 1249/4000000,
    #          m_hat = (1/50)/(1 - 81/100) = 2/19,
    #          v_hat = (1249/4000000)/(1 - 998001/1000000) = 1249/7996,
    #          theta -= (1/10)(2/19)/(sqrt(1249/7996) + eps)
    # Swapping beta1 and beta2, or dropping a bias correction, changes step 2.
    # (fp64 evaluation: 1 - 0.9 is not exactly 1/10, so compare to ~1e-15.)
    eps = 1e-8
    th, m, v = mlp.adam_step(np.array([1.0]), np.array([0.5]), np.zeros(1), np.zeros(1), 1, 0.1, 0.9, 0.999, eps)
    assert abs(m[0] - 1 / 20) < 1e-15 and abs(v[0] - 1 / 4000) < 1e-17
    th1 = 1.0 - 0.1 * 0.5 / (0.5 + eps)
    assert abs(th[0] - th1) < 1e-15
    th, m, v = mlp.adam_step(th, np.array([-0.25]), m, v, 2, 0.1, 0.9, 0.999, eps)
    assert abs(m[0] - 1 / 50) < 1e-15 and abs(v[0] - 1249 / 4000000) < 1e-17
    th2 = th1 - 0.1 * (2 / 19) / (np.sqrt(1249 / 7996) + eps)
    assert abs(th[0] - th2) < 1e-14, (th[0], th2)


def test_adam_first_step_is_lr_times_sign_for_every_parameter():
    # With zero moments, bias correction makes the first step lr * g / (|g| + eps).
    g = np.array([3.0, -2e-3, 0.0, 7.5e4])
    th, _, _ = mlp.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 0.01, 0.8, 0.99, 1e-8)
    np.testing.assert_allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
