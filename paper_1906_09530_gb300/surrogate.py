"""Warm start of low-temperature runs from a learned equilibrium interface profile.

The network (lbm_mlp_* of the C ABI, trained by this library's own kernels)
maps (T_r, kappa-hat, k, 1/R) to the equilibrium state of one interface as the
method itself settles it, including its bulk offsets from Maxwell: a flat
interface (1/R = 0) or a drop of radius R.  One surrogate is trained per
geometry (the method's drop and slab equilibria differ by far more than the
Laplace shift: the orientation effect of the discretisation).  That state,
mapped onto a slab or a drop, starts a run close to its equilibrium, so most of
the slow relaxation of the bulk densities (Sec. 5.6: the initialisation causes
the long transients at low T) is skipped.  Where the prediction is poor the
plain run still converges: the method itself is the fallback, and its own
equilibrium is what the prediction is checked against.

  * training data: flat interfaces (periodic slabs) or drops, run to
    equilibrium as one batch; each gives its bulk gas and liquid densities and
    the 236 nodes centred on its interface (the midpoint crossing, located to
    a fraction of a node; for a drop, of the azimuthally averaged radial
    profile);
  * outputs: 16 copies of 2 ln(rho_g / rho_g,Maxwell) and 4 copies of
    1000 ln(rho_l / rho_l,Maxwell), the bulk offsets, averaged on prediction
    (the copies weight them in the mean-squared loss, which otherwise the 236
    shape outputs would dominate, and average the BF16 output noise), then the
    interface shape u = (ln rho - ln rho_g) / (ln rho_l - ln rho_g) between the
    equilibrium bulks at 236 positions;
  * inputs: (T_r, kappa-hat, k, 1/R) scaled to [-1, 1] on the ranges the
    surrogate is trained for (a range of zero width maps to 0).
"""
import math

import numpy as np

from . import workloads as W
from ._binding import Batch, Mlp, lbm_maxwell

NG, NL = 16, 4  # output copies of the gas and liquid offsets
WINDOW = 256 - NG - NL
S = np.arange(WINDOW) - (WINDOW - 1) / 2.0  # window positions about the interface
G_SCALE, L_SCALE = 2.0, 1000.0
SIZES = (4, 256, 256, 256, NG + NL + WINDOW)
DEFAULT_RANGES = {"T_r": (0.35, 0.85), "kappa": (0.05, 0.15), "k": (0.1, 0.25)}


def scale_inputs(T_r, kappa, k, ranges, inv_r=None, inv_r_range=(0.0, 0.0)):
    """The network's inputs: (T_r, kappa-hat, k) on `ranges` and 1/R on
    inv_r_range, each mapped to [-1, 1] (0 for a range of zero width); inv_r
    None: flat interfaces (1/R = 0)."""
    T_r = np.asarray(T_r, dtype=np.float64)
    if inv_r is None:
        inv_r = np.zeros_like(T_r)
    cols = []
    for v, (lo, hi) in zip((T_r, kappa, k, inv_r), list(ranges.values()) + [inv_r_range]):
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


def extract_drop(rho, radius):
    """(bulk gas, bulk liquid, window) of a drop of about the given radius at the
    centre of the periodic field rho [n][n]: the gas over the outer n/16 of every
    side, the liquid over r < radius / 2, and the window from the azimuthal mean
    of rho in bins of a quarter node, about the radius where that mean crosses
    the midpoint (d = r0 - r > 0 inside the liquid; beyond the measured radii
    the bulks)."""
    n = rho.shape[0]
    b = max(n // 16, 1)
    edge = np.zeros_like(rho, dtype=bool)
    edge[:b, :] = edge[-b:, :] = edge[:, :b] = edge[:, -b:] = True
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    r = np.hypot(xx - n / 2.0, yy - n / 2.0)
    g = float(rho[edge].mean())
    l = float(rho[r < radius / 2].mean())
    rmax = n / 2.0 - 1.0
    inside = r < rmax
    bins = np.floor(r[inside] * 4).astype(int)
    cnt = np.bincount(bins)
    prof = np.bincount(bins, weights=rho[inside]) / np.maximum(cnt, 1)
    rb = (np.arange(prof.size) + 0.5) / 4
    ok = cnt > 0
    rb, prof = rb[ok], prof[ok]
    mid = 0.5 * (g + l)
    j = int(np.argmax((rb > radius / 2) & (prof < mid)))  # first bin below the midpoint
    r0 = rb[j - 1] + (mid - prof[j - 1]) * (rb[j] - rb[j - 1]) / (prof[j] - prof[j - 1])
    window = np.interp(r0 - S, rb, prof, left=l, right=g)
    return g, l, window


def drop_profiles(T_r, kappa, k, radius, n, steps, eos=None, tau=1.0):
    """Run one drop per input point (radius[i] at the centre of an n[i] x n[i]
    periodic grid, from the tanh start between the Maxwell densities) for
    `steps` steps as one batch; returns (bulk gas [m], bulk liquid [m],
    windows [m, WINDOW]) by extract_drop."""
    specs = [dict(nx=int(m), ny=int(m), T_r=float(a), kappa=float(b), k=float(c), tau=tau)
             for a, b, c, m in zip(T_r, kappa, k, n)]
    bt = Batch(specs, eos=eos)
    for i, d in enumerate(specs):
        rg, rl = lbm_maxwell(d["T_r"], eos)
        bt.set_fields(i, W.drop(d["nx"], d["ny"], rg, rl, float(radius[i]), 4.0 / d["k"]))
    bt.step(steps)
    res = [extract_drop(bt.fields(i)[0], float(radius[i])) for i in range(len(specs))]
    bt.close()
    return (np.array([x[0] for x in res]), np.array([x[1] for x in res]),
            np.stack([x[2] for x in res]))


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

    def __init__(self, seed=0, ranges=DEFAULT_RANGES, max_batch=1024, eos=None,
                 inv_r_range=(0.0, 0.0)):
        self.net = Mlp(max_batch)
        self.net.set_params(glorot_params(seed))
        self.ranges = dict(ranges)
        self.inv_r_range = tuple(inv_r_range)
        self.max_batch = max_batch
        self.eos = eos

    def fit(self, T_r, kappa, k, gas, liq, windows, epochs=200, lr=1e-3, batch=256, seed=0,
            inv_r=None):
        """Minibatch Adam on (inputs, targets), the rate decaying tenfold over
        the epochs; returns the final loss over the whole set.  inv_r: 1/R of
        each drop (None: flat interfaces)."""
        import torch
        x = scale_inputs(T_r, kappa, k, self.ranges, inv_r, self.inv_r_range)
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

    def predict(self, T_r, kappa, k, inv_r=None):
        """Predicted (bulk gas [n], bulk liquid [n], windows [n, WINDOW])."""
        import torch
        T_r, kappa, k = (np.atleast_1d(np.asarray(v, dtype=np.float64)) for v in (T_r, kappa, k))
        if inv_r is not None:
            inv_r = np.atleast_1d(np.asarray(inv_r, dtype=np.float64))
        x = scale_inputs(T_r, kappa, k, self.ranges, inv_r, self.inv_r_range)
        y = self.net.forward(torch.from_numpy(x).cuda())
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
    the window (radial distance measured outward: gas side negative), and the
    bulk liquid in its core r < radius / 2 (where extract_drop measures it; a
    small drop's core lies inside the window, whose far liquid side is the
    least certain part of a prediction)."""
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.hypot(xx - nx / 2.0, yy - ny / 2.0)
    rho = profile_at(gas, liq, window, radius - r)
    rho[r < radius / 2] = liq
    return rho


def drop_radius_for_mass(nx, ny, mass, gas, liq, window, radius):
    """The radius whose drop_field holds the given total mass (bisection about
    `radius`): a warm start of the same system as a given start field.  A
    drop's equilibrium depends on its mass (through its radius and Laplace
    pressure), so fields of different masses settle to different states."""
    lo, hi = 0.5 * radius, 1.5 * radius
    for _ in range(48):
        mid = 0.5 * (lo + hi)
        if drop_field(nx, ny, mid, gas, liq, window).sum() < mass:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


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


def settle_step(times, samples, target, rtol, window):
    """The first time at which the mean of the last `window` samples (and every
    later such mean) is within rtol (relative, elementwise) of target; None if
    the record never settles.  samples[i] is a tuple of values taken at times[i]
    (the windowed mean filters the acoustic oscillation of the bulks)."""
    v = np.asarray(samples, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    good = []
    for i in range(len(v)):
        if i + 1 < window:
            good.append(False)
            continue
        m = v[i + 1 - window:i + 1].mean(axis=0)
        good.append(bool(np.all(np.abs(m / target - 1) <= rtol)))
    for i in range(len(good)):
        if all(good[i:]):
            return times[i] if good[i] else None
    return None
