"""The surrogate network of the warm start, plain FP64 numpy: forward pass,
backward pass and Adam step, written out layer by layer.

TEST INFRASTRUCTURE ONLY (part of the oracle): only the tests and the
benchmark's CPU legs use it.  Shares no code with the CUDA library.

Network (4 layers, width 256): x[4] -> tanh(x W1 + b1) -> tanh(. W2 + b2) ->
tanh(. W3 + b3) -> . W4 + b4 = y[256].  Row vectors; W_l is [fan_in, fan_out].
Loss: mean squared error over the batch and the 256 outputs,
L = sum((y - t)^2) / (B * 256).  Adam (Kingma and Ba, 2015) with bias
correction: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
p -= lr (m / (1 - b1^s)) / (sqrt(v / (1 - b2^s)) + eps) at step s.

Parameters travel as one flat float vector in the order W1, b1, W2, b2, W3,
b3, W4, b4, each W row-major [fan_in][fan_out].

forward_rounded / loss_and_grad_rounded are the same chain rule with the
operands of every matrix product rounded first (to BF16 by default: 8
significant bits, round to nearest, ties to even), the products and everything
else still in FP64.  They define what a network whose products take BF16
operands computes, up to the accumulation and activation rounding of its own
arithmetic, so that such a network can be compared with it entry by entry.
"""
import numpy as np

SIZES = (4, 256, 256, 256, 256)
N_LAYERS = len(SIZES) - 1


def n_params():
    return sum(a * b + b for a, b in zip(SIZES[:-1], SIZES[1:]))


def unpack(p):
    """List of (W, b) views of the flat parameter vector."""
    out, o = [], 0
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        W = p[o:o + a * b].reshape(a, b)
        o += a * b
        bias = p[o:o + b]
        o += b
        out.append((W, bias))
    return out


def init_params(seed):
    """Glorot-uniform weights, zero biases, from numpy's seeded generator."""
    rng = np.random.default_rng(seed)
    parts = []
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        lim = np.sqrt(6.0 / (a + b))
        parts.append(rng.uniform(-lim, lim, size=a * b))
        parts.append(np.zeros(b))
    return np.concatenate(parts)


def bf16(x):
    """x rounded to the nearest BF16 value (8 significant bits), ties to even,
    exactly from FP64 (no intermediate FP32 rounding).  Zero stays zero."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)  # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)


def _identity(x):
    return np.asarray(x, dtype=np.float64)


def forward(p, x, rnd=_identity):
    """Outputs y [B, 256] and the activations of every layer (for backward).
    rnd is applied to both operands of every product (identity: plain FP64)."""
    acts = [np.asarray(x, dtype=np.float64)]
    layers = unpack(np.asarray(p, dtype=np.float64))
    for l, (W, b) in enumerate(layers):
        z = rnd(acts[-1]) @ rnd(W) + b
        acts.append(np.tanh(z) if l < N_LAYERS - 1 else z)
    return acts[-1], acts


def forward_rounded(p, x, rnd=bf16):
    """forward() with the operands of each product rounded by rnd."""
    return forward(p, x, rnd)


def loss_and_grad(p, x, t, rnd=_identity, parts=False):
    """Mean-squared-error loss and its gradient with respect to every parameter
    (flat, the order of the parameter vector), by the chain rule.  rnd is applied
    to both operands of every product, forward and backward (identity: plain
    FP64); the bias gradients sum the unrounded signal.  With parts=True also
    returns y, the activations and the backward signal entering each layer."""
    p = np.asarray(p, dtype=np.float64)
    y, acts = forward(p, x, rnd)
    B = y.shape[0]
    diff = y - t
    loss = float(np.sum(diff * diff) / (B * y.shape[1]))
    layers = unpack(p)
    grads = [None] * N_LAYERS
    signals = [None] * N_LAYERS
    d = 2.0 * diff / (B * y.shape[1])  # dL/dy
    for l in range(N_LAYERS - 1, -1, -1):
        W, _ = layers[l]
        signals[l] = d  # dL/dz of layer l
        grads[l] = (rnd(acts[l]).T @ rnd(d), d.sum(axis=0))
        if l > 0:
            d = (rnd(d) @ rnd(W).T) * (1.0 - acts[l] ** 2)  # through the tanh of layer l-1
    g = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    if parts:
        return loss, g, y, acts, signals
    return loss, g


def loss_and_grad_rounded(p, x, t, rnd=bf16, parts=False):
    """loss_and_grad() with the operands of each product rounded by rnd."""
    return loss_and_grad(p, x, t, rnd, parts)


def adam(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1**step)
    vh = v / (1 - b2**step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
