"""Pins of the oracle's surrogate network (oracle/mlp.py).

  * the gradient of the loss equals central finite differences of the loss
    itself, parameter by parameter, in every layer (a dropped tanh derivative,
    a transposed operand or a wrong bias sum fails);
  * with all weights zero the output is the last bias, and the loss gradient of
    that bias is 2 (b - mean target) / 256;
  * a single linear layer's gradient matches the closed form x^T (2 (y - t)/(BN));
  * one Adam step from zero moments moves each parameter by lr sign(g) (up to
    eps), the known first-step behaviour;
  * the parameter count of 3-256-256-256-256 is 198 400.
"""
import numpy as np
import pytest

from oracle import mlp


def test_parameter_count():
    assert mlp.n_params() == 3 * 256 + 256 + 3 * (256 * 256 + 256) == 198400


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = mlp.init_params(11)
    x = rng.uniform(-1, 1, (5, 3))
    t = rng.uniform(-1, 1, (5, 256))
    _, g = mlp.loss_and_grad(p, x, t)
    # sample parameters from every layer's weights and biases
    offs, o = [], 0
    for a, b in zip(mlp.SIZES[:-1], mlp.SIZES[1:]):
        offs += list(o + rng.choice(a * b, 6, replace=False))
        o += a * b
        offs += list(o + rng.choice(b, 3, replace=False))
        o += b
    h = 1e-6
    for i in offs:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_and_grad(pp, x, t)[0] - mlp.loss_and_grad(pm, x, t)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-10), i


def test_zero_weights_give_last_bias():
    p = np.zeros(mlp.n_params())
    b4 = np.linspace(-1, 1, 256)
    p[-256:] = b4
    x = np.ones((4, 3))
    y, _ = mlp.forward(p, x)
    assert np.array_equal(y, np.tile(b4, (4, 1)))
    t = np.random.default_rng(1).uniform(size=(4, 256))
    _, g = mlp.loss_and_grad(p, x, t)
    assert np.allclose(g[-256:], 2 * (b4 - t.mean(axis=0)) / 256, rtol=1e-13)


def test_linear_layer_closed_form():
    """Only the last layer varies (the hidden activations are fixed): its weight
    gradient is a^T (2 (y - t) / (B N)) with a the last hidden activation."""
    rng = np.random.default_rng(5)
    p = mlp.init_params(2)
    x = rng.uniform(-1, 1, (7, 3))
    t = rng.uniform(-1, 1, (7, 256))
    y, acts = mlp.forward(p, x)
    _, g = mlp.loss_and_grad(p, x, t)
    gw4 = g[-256 * 256 - 256:-256].reshape(256, 256)
    assert np.allclose(gw4, acts[3].T @ (2 * (y - t) / (7 * 256)), rtol=1e-12, atol=1e-15)


def test_adam_first_step():
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = mlp.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 1e-3)
    assert np.allclose(p, -1e-3 * np.sign(g), rtol=1e-4)
