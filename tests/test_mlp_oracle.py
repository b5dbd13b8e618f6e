"""Pins for the fp64 MLP oracle: finite differences and closed forms."""
import numpy as np

from oracle import mlp


def small_problem(seed=0, B=7):
    rng = np.random.default_rng(seed)
    p = mlp.init_params(seed)
    X = rng.uniform(-1, 1, (B, 4))
    T = rng.uniform(-1, 1, (B, 3))
    return p, X, T


def test_gradients_match_central_differences():
    p, X, T = small_problem()
    _, g = mlp.backward(p, X, T)
    rng = np.random.default_rng(1)
    for key, shape in mlp.SHAPES:
        for _ in range(6):
            idx = tuple(int(rng.integers(0, s)) for s in shape)
            num = mlp.numeric_grad(p, X, T, key, idx)
            assert abs(num - g[key][idx]) <= 1e-6 * max(1.0, abs(num)), (key, idx)


def test_output_layer_closed_form():
    # with W3 = 0 the output is b3 for every sample and dL/db3 = 2 mean(b3 - t)/O
    p, X, T = small_problem(2)
    p["W3"][:] = 0.0
    p["b3"] = np.array([0.5, -0.25, 1.0])
    L, g = mlp.backward(p, X, T)
    assert np.isclose(L, np.mean((p["b3"] - T) ** 2))
    np.testing.assert_allclose(g["b3"], 2.0 * (p["b3"] - T).mean(axis=0) / 3.0)
    assert np.all(g["W2"] == 0) and np.all(g["W1"] == 0)


def test_dead_relu_gives_zero_hidden_grads():
    p, X, T = small_problem(3)
    p["b1"][:] = -100.0
    _, g = mlp.backward(p, X, T)
    assert np.all(g["W1"] == 0) and np.all(g["b1"] == 0) and np.all(g["W2"] == 0)


def test_adam_first_step_is_lr_times_sign():
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -4.0, 1e-3])}
    mlp.adam_step(p, g, {}, t=1, lr=0.01, eps=1e-12)
    np.testing.assert_allclose(p["w"], [1.0 - 0.01, -2.0 + 0.01, 3.0 - 0.01], rtol=1e-9)


def test_training_reduces_loss():
    p, X, T = small_problem(4, B=32)
    state = {}
    L0 = mlp.loss(p, X, T)
    for t in range(1, 301):
        _, g = mlp.backward(p, X, T)
        mlp.adam_step(p, g, state, t, lr=3e-3)
    assert mlp.loss(p, X, T) < 0.2 * L0
