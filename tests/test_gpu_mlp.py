"""The surrogate network's kernels (lbm_mlp_* of the C ABI) against the FP64
oracle (oracle/mlp.py, pinned by test_oracle_mlp.py), on the same float32
parameters and inputs.

Tolerances come from the arithmetic: every product takes BF16 operands (8
significant bits, unit 2^-8 = 3.9e-3) with FP32 accumulation over K <= 256 terms
whose rounding errors add up like a random walk, through four layers.  Relative
L2 errors of about 1e-2 are expected, and the bounds are 2e-2 (outputs) and 5e-2
(each layer's gradient), with the gradient's direction within 0.1% (cosine).

Entry by entry the kernels are compared with the oracle's rounded network
(oracle.mlp.loss_and_grad_rounded), which takes the same BF16 operands in every
product.  What separates the two is FP32 accumulation and activation rounding,
and the rare BF16 rounding that lands on the other side of a tie because the
activation or signal feeding it differs in its last FP32 bits.  Each entry's
bound is c times its BF16 scale: one BF16 unit (2^-8) on each of the K terms of
its product, added in quadrature, plus the scale of the signal it was built
from.  A CPU stand-in of the same arithmetic stays below 2.0 of the scale; a
single weight off by 0.02 gives 5 to 60.  c = 4.
"""
import numpy as np
import pytest

from oracle import mlp as O

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _setup(cuda, B, seed=4):
    from paper_1906_09530_gb300 import Mlp
    torch = cuda
    rng = np.random.default_rng(seed)
    p = O.init_params(seed).astype(np.float32)
    x = rng.uniform(-1, 1, (B, 4)).astype(np.float32)
    t = (0.5 + 0.4 * np.sin(np.outer(x[:, 0] + 0.5 * x[:, 1] - x[:, 2], np.linspace(0, 3, 256)))
         ).astype(np.float32)
    net = Mlp(max_batch=max(512, B))
    net.set_params(p)
    return net, p, x, t, torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()


U8 = 2.0 ** -8
C_BOUND = 4.0


def _scales(p, x, t):
    """The rounded network's outputs and gradient with each entry's BF16 scale."""
    p = np.asarray(p, np.float64)
    layers = O.unpack(p)
    _, g, y, acts, sig = O.loss_and_grad_rounded(p, x, t, parts=True)
    W4 = O.bf16(layers[-1][0])
    sy = U8 * np.sqrt((O.bf16(acts[-2]) ** 2) @ (W4 ** 2))
    B, N = y.shape
    sd = 2.0 / (B * N) * sy  # scale of dL/dy
    out = [None] * O.N_LAYERS
    for l in range(O.N_LAYERS - 1, -1, -1):
        qa, qd = O.bf16(acts[l]), O.bf16(sig[l])
        sW = U8 * np.sqrt((qa ** 2).T @ (qd ** 2)) + np.sqrt((qa ** 2).T @ (sd ** 2))
        out[l] = (sW, np.sqrt((sd ** 2).sum(0)))
        if l > 0:
            qW = O.bf16(layers[l][0])
            sd = (U8 * np.sqrt((qd ** 2) @ (qW.T ** 2)) + np.sqrt((sd ** 2) @ (qW.T ** 2))) \
                * np.abs(1 - acts[l] ** 2)
    sg = np.concatenate([np.concatenate([a.ravel(), b]) for a, b in out])
    return y, sy, g, sg


def test_paths_agree_closely(cuda):
    """tcgen05 and mma.sync take the same BF16 operands and accumulate in FP32:
    their outputs differ only by the order of the FP32 additions."""
    net, p, x, t, dx, dt = _setup(cuda, 300)
    y_tc = net.forward(dx).cpu().numpy()
    net.tcgen05 = False
    y_ms = net.forward(dx).cpu().numpy()
    assert np.abs(y_tc - y_ms).max() <= 2e-3 * np.abs(y_ms).max()


def test_batch_size_changes(cuda):
    """One network called with batch sizes in turn (the tensor maps are made
    again for each new size) gives what fresh networks give, bit for bit."""
    from paper_1906_09530_gb300 import Mlp
    net, p, x, t, dx, dt = _setup(cuda, 300)
    got = {}
    for B in (300, 37, 300, 129):
        got.setdefault(B, []).append(net.forward(dx[:B].contiguous()).cpu().numpy())
        got.setdefault(("g", B), []).append(
            net.loss_grad(dx[:B].contiguous(), dt[:B].contiguous())[1].cpu().numpy())
    for B in (300, 37, 129):
        fresh = Mlp(max_batch=512)
        fresh.set_params(p)
        y = fresh.forward(dx[:B].contiguous()).cpu().numpy()
        g = fresh.loss_grad(dx[:B].contiguous(), dt[:B].contiguous())[1].cpu().numpy()
        for a in got[B]:
            assert np.array_equal(a, y)
        for a in got[("g", B)]:
            assert np.array_equal(a, g)


def test_params_round_trip(cuda):
    net, p, *_ = _setup(cuda, 8)
    assert np.array_equal(net.get_params(), p)
    assert net.n_params == O.n_params()


@pytest.mark.parametrize("B", [1, 37, 300])
def test_forward_matches_oracle(cuda, B):
    net, p, x, t, dx, dt = _setup(cuda, B)
    y = net.forward(dx).cpu().numpy()
    y_ref, _ = O.forward(p.astype(np.float64), x.astype(np.float64))
    assert _rel(y, y_ref) <= 2e-2


def test_tcgen05_path_in_use(cuda):
    """The forward and input-gradient products run on tcgen05 by default, and
    the switch to the mma.sync comparison kernel is the caller's to make."""
    net, p, x, t, dx, dt = _setup(cuda, 8)
    assert net.tcgen05
    net.forward(dx)
    net.loss_grad(dx, dt)
    assert net.tcgen05  # no fall back: both tensor maps were made
    net.tcgen05 = False
    assert not net.tcgen05
    net.tcgen05 = True
    assert net.tcgen05


@pytest.mark.parametrize("tc", [True, False], ids=["tcgen05", "mma_sync"])
@pytest.mark.parametrize("B", [1, 7, 37, 128, 129, 300, 512, 40000])
def test_forward_entrywise(cuda, B, tc):
    """Every output entry within C_BOUND BF16 scales of the rounded oracle: one
    row, a part of a core matrix (7), one and several 128-row tiles with
    ragged tails, and the largest batch."""
    net, p, x, t, dx, dt = _setup(cuda, B)
    net.tcgen05 = tc
    y = net.forward(dx).cpu().numpy().astype(np.float64)
    y_ref, s, _, _ = _scales(p, x.astype(np.float64), t.astype(np.float64))
    ratio = np.abs(y - y_ref) / s
    assert ratio.max() <= C_BOUND, (ratio.max(), np.unravel_index(ratio.argmax(), ratio.shape))


@pytest.mark.parametrize("tc", [True, False], ids=["tcgen05", "mma_sync"])
@pytest.mark.parametrize("B", [7, 200, 512, 5000])
def test_gradient_entrywise(cuda, B, tc):
    """Every gradient entry, weights and biases of all four layers, within
    C_BOUND BF16 scales of the rounded oracle's chain rule."""
    net, p, x, t, dx, dt = _setup(cuda, B)
    net.tcgen05 = tc
    _, g = net.loss_grad(dx, dt)
    g = g.cpu().numpy().astype(np.float64)
    _, _, g_ref, sg = _scales(p, x.astype(np.float64), t.astype(np.float64))
    ratio = np.abs(g - g_ref) / (sg + 1e-300)
    o = 0
    for l, (a, b) in enumerate(zip(O.SIZES[:-1], O.SIZES[1:])):
        for what, n in (("W", a * b), ("b", b)):
            r = ratio[o:o + n]
            assert r.max() <= C_BOUND, (l, what, r.max(), int(r.argmax()))
            o += n


def test_loss_and_gradient_match_oracle(cuda):
    net, p, x, t, dx, dt = _setup(cuda, 200)
    loss, g = net.loss_grad(dx, dt)
    g = g.cpu().numpy().astype(np.float64)
    loss_ref, g_ref = O.loss_and_grad(p.astype(np.float64), x, t)
    assert loss == pytest.approx(loss_ref, rel=2e-2)
    o = 0
    for a, b in zip(O.SIZES[:-1], O.SIZES[1:]):
        for n in (a * b, b):
            gs, rs = g[o:o + n], g_ref[o:o + n]
            assert _rel(gs, rs) <= 5e-2
            assert gs @ rs / (np.linalg.norm(gs) * np.linalg.norm(rs)) >= 0.999
            o += n


def test_adam_steps_follow_oracle(cuda):
    """Five Adam steps on the GPU against five on the oracle from the same
    start: the parameters stay within a few hundredths of the step size."""
    net, p, x, t, dx, dt = _setup(cuda, 128)
    lr = 1e-3
    for _ in range(5):
        net.train_step(dx, dt, lr)
    q = p.astype(np.float64)
    m, v = np.zeros_like(q), np.zeros_like(q)
    for s in range(1, 6):
        _, g = O.loss_and_grad(q, x, t)
        q, m, v = O.adam(q, g, m, v, s, lr)
    got = net.get_params().astype(np.float64)
    # each step moves a parameter by about lr; compare the displacements
    assert _rel(got - p, q - p) <= 5e-2


def test_training_reduces_loss(cuda):
    net, p, x, t, dx, dt = _setup(cuda, 256)
    l0 = net.train_step(dx, dt, 2e-3, want_loss=True)
    for _ in range(300):
        net.train_step(dx, dt, 2e-3)
    l1 = net.loss_grad(dx, dt)[0]
    assert l1 < 0.05 * l0
