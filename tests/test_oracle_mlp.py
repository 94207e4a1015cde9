"""Pins of the oracle's surrogate network (oracle/mlp.py).

  * the gradient of the loss equals central finite differences of the loss
    itself, parameter by parameter, in every layer (a dropped tanh derivative,
    a transposed operand or a wrong bias sum fails);
  * with all weights zero the output is the last bias, and the loss gradient of
    that bias is 2 (b - mean target) / 256;
  * a single linear layer's gradient matches the closed form x^T (2 (y - t)/(BN));
  * one Adam step from zero moments moves each parameter by lr sign(g) (up to
    eps), the known first-step behaviour;
  * the parameter count of 4-256-256-256-256 is 198 656.
"""
import numpy as np
import pytest

from oracle import mlp


def test_parameter_count():
    assert mlp.n_params() == 4 * 256 + 256 + 3 * (256 * 256 + 256) == 198656


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = mlp.init_params(11)
    x = rng.uniform(-1, 1, (5, 4))
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
    x = np.ones((4, 4))
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
    x = rng.uniform(-1, 1, (7, 4))
    t = rng.uniform(-1, 1, (7, 256))
    y, acts = mlp.forward(p, x)
    _, g = mlp.loss_and_grad(p, x, t)
    gw4 = g[-256 * 256 - 256:-256].reshape(256, 256)
    assert np.allclose(gw4, acts[3].T @ (2 * (y - t) / (7 * 256)), rtol=1e-12, atol=1e-15)


def test_adam_first_step():
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = mlp.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 1e-3)
    assert np.allclose(p, -1e-3 * np.sign(g), rtol=1e-4)


def test_bf16_rounding_matches_torch():
    """bf16() rounds as torch's float32 -> bfloat16 conversion does (nearest,
    ties to even), including exact ties and values across many binades."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    # exact ties: 8 significant bits plus a trailing half unit, both parities
    ties = np.array([1 + (2 * j + 1) / 512 for j in range(64)] + [-3.0 * (1 + 3 / 512)],
                    dtype=np.float32)
    x = np.concatenate([x, ties, np.float32([0.0, 1.0, -2.5e-30])])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x.astype(np.float64)), ref)


def test_rounded_network_matches_torch_bfloat16_casts():
    """The rounded forward and backward passes against the same chain rule
    written with torch tensors cast to bfloat16 at every product (autograd is
    not used: the rounding points are the product operands)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    p = mlp.init_params(2).astype(np.float32).astype(np.float64)
    x = rng.uniform(-1, 1, (7, 4)).astype(np.float32).astype(np.float64)
    t = rng.uniform(-1, 1, (7, 256))
    loss, g = mlp.loss_and_grad_rounded(p, x, t)

    def r(a):
        return torch.as_tensor(a).to(torch.bfloat16).to(torch.float64)
    Ws, bs, o = [], [], 0
    for a_, b_ in zip(mlp.SIZES[:-1], mlp.SIZES[1:]):
        Ws.append(torch.as_tensor(p[o:o + a_ * b_].reshape(a_, b_)))
        o += a_ * b_
        bs.append(torch.as_tensor(p[o:o + b_]))
        o += b_
    acts = [torch.as_tensor(x)]
    for l in range(4):
        z = r(acts[-1]) @ r(Ws[l]) + bs[l]
        acts.append(torch.tanh(z) if l < 3 else z)
    y = acts[-1]
    d = 2 * (y - torch.as_tensor(t)) / y.numel()
    out = []
    for l in range(3, -1, -1):
        out.append((r(acts[l]).T @ r(d), d.sum(0)))
        d = (r(d) @ r(Ws[l]).T) * (1 - acts[l] ** 2)
    g_ref = np.concatenate([np.concatenate([gw.numpy().ravel(), gb.numpy()]) for gw, gb in out[::-1]])
    assert loss == pytest.approx(float(((y - torch.as_tensor(t)) ** 2).mean()), rel=1e-14)
    assert np.allclose(g, g_ref, rtol=1e-12, atol=1e-18)
    # and the rounding is what separates it from the plain FP64 network: close
    # to it at the BF16 level, but not equal
    _, g64 = mlp.loss_and_grad(p, x, t)
    rel = np.linalg.norm(g - g64) / np.linalg.norm(g64)
    assert 1e-4 < rel < 3e-2
