"""The learned rank predictor: the oracle's FP64 network against the
mathematics (CPU), and the library's BF16 training kernels against the
oracle (GPU)."""
import numpy as np
import pytest

from oracle import mlp


def _net(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0.0, scale, mlp.N_PARAMS)
    X = rng.normal(0.0, 1.0, (40, mlp.N_IN))
    y = rng.uniform(0.0, 1.0, 40)
    return theta, X, y


def test_oracle_gradient_matches_central_differences():
    """The chain-rule gradient of the oracle's loss equals central finite
    differences of the loss (FP64, step 1e-6) to 1e-6 relative, on every
    parameter group."""
    theta, X, y = _net(1)
    loss, g = mlp.loss_and_grad(theta, X, y)
    assert abs(loss - np.mean((mlp.forward(theta, X) - y) ** 2)) <= 1e-14 * loss
    rng = np.random.default_rng(2)
    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 300, replace=False), [mlp.N_PARAMS - 1]])
    h = 1e-6
    fd = np.empty(len(idx))
    for t, k in enumerate(idx):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd[t] = (mlp.loss_and_grad(tp, X, y)[0] - mlp.loss_and_grad(tm, X, y)[0]) / (2 * h)
    assert np.abs(fd - g[idx]).max() <= 1e-6 * np.abs(g).max()


def test_oracle_gradient_closed_form_for_constant_network():
    """With zero weights and biases except b3 the network outputs b3 for
    every input: the loss is mean((b3 - y)^2), its derivative in b3 is
    2 mean(b3 - y) and every other gradient entry is 0."""
    theta = np.zeros(mlp.N_PARAMS)
    theta[-1] = 0.25
    _, X, y = _net(3)
    loss, g = mlp.loss_and_grad(theta, X, y)
    assert abs(loss - np.mean((0.25 - y) ** 2)) <= 1e-15
    assert abs(g[-1] - 2 * np.mean(0.25 - y)) <= 1e-15
    assert np.all(g[:-1] == 0.0)


def test_oracle_parameter_layout():
    p = mlp.unpack(np.arange(mlp.N_PARAMS, dtype=np.float64))
    assert mlp.N_PARAMS == 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1
    assert p["W1"][1, 0] == 16 and p["b1"][0] == 1024 and p["b3"][0] == mlp.N_PARAMS - 1
    assert np.array_equal(mlp.pack(p), np.arange(mlp.N_PARAMS))
