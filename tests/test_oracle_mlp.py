"""Pins for the oracle's selector MLP (no GPU): finite differences, closed forms, Adam."""
import numpy as np

import graphgen as gg
from oracle import mlp


def data(seed, B=9):
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 1, (B, 16))
    t = rng.normal(0, 1, (B, 4))
    mask = (rng.random((B, 4)) < 0.7).astype(np.float64)
    return x, t, mask


def test_parameter_count():
    assert mlp.N_PARAMS == 5508
    w = gg.mlp_weights(1)
    assert w.shape == (5508,)
    np.testing.assert_array_equal(mlp.pack(mlp.unpack(w)), w.astype(np.float64))


def test_gradient_matches_finite_differences():
    w = gg.mlp_weights(3).astype(np.float64)
    x, t, mask = data(4)
    g = mlp.grad(w, x, t, mask)
    rng = np.random.default_rng(5)
    idx = np.concatenate([rng.choice(1024, 40, replace=False),            # W1
                          1024 + rng.choice(64, 10, replace=False),        # b1
                          1088 + rng.choice(4096, 60, replace=False),      # W2
                          5184 + rng.choice(64, 10, replace=False),        # b2
                          5248 + np.arange(256)[::8],                      # W3
                          5504 + np.arange(4)])                            # b3
    eps = 1e-6
    for i in idx:
        wp = w.copy(); wp[i] += eps
        wm = w.copy(); wm[i] -= eps
        num = (mlp.loss(wp, x, t, mask) - mlp.loss(wm, x, t, mask)) / (2 * eps)
        assert abs(num - g[i]) <= 1e-6 + 1e-5 * abs(num), (i, num, g[i])


def test_closed_form_constant_hidden_layer():
    # W2 = 0 makes h2 = relu(b2) whatever the input, so y = relu(b2) W3 + b3
    p = mlp.unpack(gg.mlp_weights(7).astype(np.float64))
    p["W2"] = np.zeros_like(p["W2"])
    w = mlp.pack(p)
    x, _, _ = data(8)
    y, _ = mlp.forward(w, x)
    want = np.maximum(p["b2"], 0) @ p["W3"] + p["b3"]
    np.testing.assert_allclose(y, np.broadcast_to(want, y.shape), rtol=1e-12, atol=1e-12)


def test_hand_computed_tiny_network():
    # one path: x0 -> h1[0] (weight 2) -> h2[0] (weight 3) -> y[1] (weight 0.5), biases b3 = (1,0,0,0)
    p = {n: np.zeros(s) for n, s in mlp.SHAPES}
    p["W1"][0, 0] = 2.0
    p["W2"][0, 0] = 3.0
    p["W3"][0, 1] = 0.5
    p["b3"][0] = 1.0
    w = mlp.pack(p)
    x = np.zeros((2, 16)); x[0, 0] = 1.5; x[1, 0] = -1.0
    y, _ = mlp.forward(w, x)
    np.testing.assert_allclose(y, [[1.0, 4.5, 0, 0], [1.0, 0.0, 0, 0]])  # relu cuts the negative path
    t = np.zeros((2, 4)); mask = np.ones((2, 4))
    assert abs(mlp.loss(w, x, t, mask) - (1 + 4.5 ** 2 + 1) / 8) < 1e-12


def test_adam_first_step_is_signed_lr():
    w = np.zeros(5)
    g = np.array([0.3, -2.0, 1e-3, 0.0, 5.0])
    w1, m, v = mlp.adam_step(w, np.zeros(5), np.zeros(5), g, 1, 0.01)
    np.testing.assert_allclose(w1, -0.01 * np.sign(g) * (np.abs(g) / (np.abs(g) + 1e-8)), rtol=1e-9)
