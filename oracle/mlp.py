"""Plain numpy fp64 reference of the format selector's network (test infrastructure only).

16 -> 64 -> 64 -> 10 multilayer perceptron with ReLU between layers; loss
L = inv_count * sum mask * (y_hat - y)^2.  Parameters are packed as W1[16][64],
b1[64], W2[64][64], b2[64], W3[64][10], b3[10] (row-major, input index first),
the layout of include/morphstore.h.  Backpropagation is written out layer by
layer (chain rule), and tests/test_oracle_mlp.py pins it against central finite
differences of the loss.  The optimiser step is Adam (Kingma & Ba, ICLR 2015,
Algorithm 1), pinned by a two-step example worked out by hand.
"""
from __future__ import annotations

import numpy as np

IN, H, OUT = 16, 64, 10
SHAPES = [("W1", (IN, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, OUT)), ("b3", (OUT,))]
PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)  # 5898


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


def pack(p) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def forward(theta, x):
    """Returns the output y_hat[n][10] and the hidden activations."""
    p = unpack(theta)
    x = np.asarray(x, dtype=np.float64)
    a1 = x @ p["W1"] + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ p["W3"] + p["b3"]
    return y, (x, a1, h1, a2, h2)


def loss(theta, x, y, mask, inv_count) -> float:
    yh, _ = forward(theta, x)
    e = (yh - np.asarray(y, np.float64)) * np.asarray(mask, np.float64)
    return float(inv_count * np.sum(e * e))


def loss_grad(theta, x, y, mask, inv_count):
    """(L, dL/dtheta) by backpropagation."""
    p = unpack(theta)
    yh, (x, a1, h1, a2, h2) = forward(theta, x)
    m = np.asarray(mask, np.float64)
    e = (yh - np.asarray(y, np.float64)) * m
    L = float(inv_count * np.sum(e * e))
    dy = 2.0 * inv_count * e * m           # dL/dy_hat
    g = {"W3": h2.T @ dy, "b3": dy.sum(axis=0)}
    dh2 = dy @ p["W3"].T
    da2 = dh2 * (a2 > 0)
    g["W2"] = h1.T @ da2
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ p["W2"].T
    da1 = dh1 * (a1 > 0)
    g["W1"] = x.T @ da1
    g["b1"] = da1.sum(axis=0)
    return L, pack(g)


def adam_step(theta, grad, m, v, step, lr, beta1, beta2, eps):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) in fp64; returns new
    (theta, m, v).  In the paper's order: the biased first and second moment
    estimates are decayed and updated with the gradient, both are divided by their
    bias corrections 1 - beta^t, and the parameters move by lr times the corrected
    first moment over (the root of the corrected second moment plus eps)."""
    g = np.asarray(grad, np.float64)
    m_t = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v_t = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    m_hat = m_t / (1.0 - beta1 ** step)
    v_hat = v_t / (1.0 - beta2 ** step)
    theta_t = np.asarray(theta, np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps)
    return theta_t, m_t, v_t


def init(seed: int) -> np.ndarray:
    """He-style initialisation from a seeded generator (biases zero)."""
    rng = np.random.default_rng(seed)
    p = {"W1": rng.normal(0, np.sqrt(2.0 / IN), (IN, H)), "b1": np.zeros(H),
         "W2": rng.normal(0, np.sqrt(2.0 / H), (H, H)), "b2": np.zeros(H),
         "W3": rng.normal(0, np.sqrt(1.0 / H), (H, OUT)), "b3": np.zeros(OUT)}
    return pack(p)
