"""Warm start of low-temperature runs from a learned equilibrium interface profile.

The network (lbm_mlp_* of the C ABI, trained by this library's own kernels)
maps (T_r, kappa-hat, k) to the equilibrium state of one flat interface as the
method itself settles it, including its offsets from Maxwell.  That state,
mapped onto a slab or a drop, starts a run close to its equilibrium, so most of
the slow relaxation of the bulk densities (Sec. 5.6: the initialisation causes
the long transients at low T) is skipped.  Where the prediction is poor the
plain run still converges: the method itself is the fallback, and its own
equilibrium is what the prediction is checked against.

  * training data: flat interfaces (periodic slabs) run to equilibrium as one
    batch; each gives its bulk gas and liquid densities and the 236 nodes
    centred on its lower interface (the midpoint crossing, located to a
    fraction of a node);
  * outputs: 16 copies of 2 ln(rho_g / rho_g,Maxwell) and 4 copies of
    1000 ln(rho_l / rho_l,Maxwell), the bulk offsets, averaged on prediction
    (the copies weight them in the mean-squared loss, which otherwise the 236
    shape outputs would dominate, and average the BF16 output noise), then the
    interface shape u = (ln rho - ln rho_g) / (ln rho_l - ln rho_g) between the
    equilibrium bulks at 236 positions;
  * inputs: (T_r, kappa-hat, k) scaled to [-1, 1] on the ranges the surrogate
    is trained for.
"""
import math

import numpy as np

from . import workloads as W
from ._binding import Batch, Mlp, lbm_maxwell

NG, NL = 16, 4  # output copies of the gas and liquid offsets
WINDOW = 256 - NG - NL
S = np.arange(WINDOW) - (WINDOW - 1) / 2.0  # window positions about the interface
G_SCALE, L_SCALE = 2.0, 1000.0
SIZES = (3, 256, 256, 256, NG + NL + WINDOW)
DEFAULT_RANGES = {"T_r": (0.35, 0.85), "kappa": (0.05, 0.15), "k": (0.1, 0.25)}


def scale_inputs(T_r, kappa, k, ranges):
    cols = []
    for v, (lo, hi) in zip((T_r, kappa, k), ranges.values()):
        mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
        cols.append((np.asarray(v, dtype=np.float64) - mid) / (half if half > 0 else 1.0))
    return np.stack(cols, axis=-1).astype(np.float32)


def sample_inputs(n, seed, ranges=DEFAULT_RANGES):
    """n points of the input box, uniform, from splitmix64 of (seed, index)."""
    idx = np.arange(3 * n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        key = W.splitmix64(np.uint64(seed) * np.uint64(0x100000001B3) + idx)
    u = ((key >> np.uint64(11)).astype(np.float64) / 9007199254740992.0).reshape(n, 3)
    return tuple(lo + (hi - lo) * u[:, j] for j, (lo, hi) in enumerate(ranges.values()))


def extract(r):
    """(bulk gas, bulk liquid, window) of a flat slab column r (liquid in the
    middle, interfaces near ny/4 and 3ny/4): bulk means over the central fifth
    of each phase, and the densities at the window positions about the lower
    interface by linear interpolation."""
    ny = r.size
    g = np.r_[r[: ny // 10], r[-ny // 10:]].mean()
    l = r[ny // 2 - ny // 10: ny // 2 + ny // 10].mean()
    half = r[: ny // 2]
    mid = 0.5 * (g + l)
    i = int(np.argmax(half >= mid))  # first node at or above the midpoint
    y0 = (i - 1) + (mid - r[i - 1]) / (r[i] - r[i - 1])
    pos = (y0 + S) % ny
    lo = np.floor(pos).astype(int)
    w = pos - lo
    return g, l, (1 - w) * r[lo % ny] + w * r[(lo + 1) % ny]


def to_target(g, l, window, rg, rl):
    u = (np.log(window) - math.log(g)) / (math.log(l) - math.log(g))
    return np.concatenate([np.full(NG, G_SCALE * math.log(g / rg)),
                           np.full(NL, L_SCALE * math.log(l / rl)), u])


def from_target(t, rg, rl):
    """(bulk gas, bulk liquid, window densities) from a network output."""
    g = rg * math.exp(float(np.mean(t[:NG])) / G_SCALE)
    l = rl * math.exp(float(np.mean(t[NG:NG + NL])) / L_SCALE)
    u = np.clip(t[NG + NL:], 0.0, 1.0)
    return g, l, np.exp(math.log(g) + u * (math.log(l) - math.log(g)))


def equilibrium_profiles(T_r, kappa, k, steps, ny=384, eos=None, tau=1.0):
    """Run one flat slab per input point for `steps` steps as one batch;
    returns (bulk gas [n], bulk liquid [n], windows [n, WINDOW])."""
    specs = [dict(nx=8, ny=ny, T_r=float(a), kappa=float(b), k=float(c), tau=tau)
             for a, b, c in zip(T_r, kappa, k)]
    b = Batch(specs, eos=eos)
    for i, d in enumerate(specs):
        rg, rl = lbm_maxwell(d["T_r"], eos)
        b.set_fields(i, W.flat(8, ny, rg, rl, ny / 2, 4.0 / d["k"]))
    b.step(steps)
    res = [extract(b.fields(i)[0][:, 0]) for i in range(len(specs))]
    b.close()
    return (np.array([x[0] for x in res]), np.array([x[1] for x in res]),
            np.stack([x[2] for x in res]))


def glorot_params(seed):
    """Glorot-uniform weights and zero biases in the library's parameter order."""
    rng = np.random.default_rng(seed)
    parts = []
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        lim = math.sqrt(6.0 / (a + b))
        parts.append(rng.uniform(-lim, lim, size=a * b))
        parts.append(np.zeros(b))
    return np.concatenate(parts).astype(np.float32)


class Surrogate:
    """The network, the input ranges it is trained for, and the EOS whose
    Maxwell pairs its outputs are read against."""

    def __init__(self, seed=0, ranges=DEFAULT_RANGES, max_batch=1024, eos=None):
        self.net = Mlp(max_batch)
        self.net.set_params(glorot_params(seed))
        self.ranges = dict(ranges)
        self.max_batch = max_batch
        self.eos = eos

    def fit(self, T_r, kappa, k, gas, liq, windows, epochs=200, lr=1e-3, batch=256, seed=0):
        """Minibatch Adam on (inputs, targets), the rate decaying tenfold over
        the epochs; returns the final loss over the whole set."""
        import torch
        x = scale_inputs(T_r, kappa, k, self.ranges)
        t = np.stack([to_target(g, l, w, *lbm_maxwell(float(a), self.eos))
                      for g, l, w, a in zip(gas, liq, windows, T_r)]).astype(np.float32)
        dx, dt = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
        n = len(x)
        batch = min(batch, n)
        rng = np.random.default_rng(seed)
        for e in range(epochs):
            order = torch.from_numpy(rng.permutation(n)).cuda()
            rate = lr * (0.1 ** (e / max(epochs - 1, 1)))
            for s in range(0, n - batch + 1, batch):
                idx = order[s:s + batch]
                self.net.train_step(dx[idx].contiguous(), dt[idx].contiguous(), rate)
        loss = 0.0
        for s in range(0, n, self.max_batch):
            m = min(self.max_batch, n - s)
            loss += self.net.loss_grad(dx[s:s + m], dt[s:s + m])[0] * m
        return loss / n

    def predict(self, T_r, kappa, k):
        """Predicted (bulk gas [n], bulk liquid [n], windows [n, WINDOW])."""
        import torch
        T_r, kappa, k = (np.atleast_1d(np.asarray(v, dtype=np.float64)) for v in (T_r, kappa, k))
        y = self.net.forward(torch.from_numpy(scale_inputs(T_r, kappa, k, self.ranges)).cuda())
        y = y.cpu().numpy().astype(np.float64)
        out = [from_target(y[i], *lbm_maxwell(float(T_r[i]), self.eos)) for i in range(len(T_r))]
        return (np.array([o[0] for o in out]), np.array([o[1] for o in out]),
                np.stack([o[2] for o in out]))

    def close(self):
        self.net.close()


def profile_at(gas, liq, window, d):
    """Density at signed distance d from the interface (d < 0 on the gas
    side): the window inside it, the bulk values beyond its ends."""
    return np.interp(d, S, window, left=gas, right=liq)


def flat_field(nx, ny, gas, liq, window):
    """A slab (liquid in the middle, interfaces at ny/4 and 3ny/4) whose
    interfaces carry the window."""
    y = np.arange(ny, dtype=np.float64)
    d = ny / 4.0 - np.abs(y - ny / 2.0)  # > 0 inside the liquid
    return np.repeat(profile_at(gas, liq, window, d)[:, None], nx, axis=1)


def drop_field(nx, ny, radius, gas, liq, window):
    """A drop of the given radius at the domain centre whose interface carries
    the window (radial distance measured outward: gas side negative)."""
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.hypot(xx - nx / 2.0, yy - ny / 2.0)
    return profile_at(gas, liq, window, radius - r)


def steps_to_equilibrium(sim, probe, target, rtol, every=500, max_steps=2_000_000):
    """Steps until probe(sim) is within rtol (relative, elementwise) of target,
    checked every `every` steps; None if not reached by max_steps."""
    target = np.asarray(target, dtype=np.float64)
    while sim.t < max_steps:
        v = np.asarray(probe(sim), dtype=np.float64)
        if np.all(np.abs(v / target - 1) <= rtol):
            return sim.t
        sim.step(every)
    return None
