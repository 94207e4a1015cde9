"""Host-side helpers on known inputs, without a GPU.

  * the seeded input generator (shared by the CUDA path and the oracle, none of
    the method's arithmetic) reproduces splitmix64's published outputs
    (tests/golden/splitmix64.json), and its noise is in range and can be
    recomputed node by node;
  * the warm start's target encoding (bulk offsets from Maxwell in log space,
    the interface shape between the bulks) round-trips, and its interface
    extraction recovers a window laid onto a slab;
  * the input scaling maps each range onto [-1, 1];
  * the equilibrium stopping rule stops at the first check within tolerance.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1906_09530_gb300 import surrogate as S
from paper_1906_09530_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.json")


def test_splitmix64_published_outputs():
    d = json.load(open(GOLDEN))
    gamma = np.uint64(int(d["gamma"], 16))
    for seq in d["sequences"]:
        n = len(seq["outputs"])
        with np.errstate(over="ignore"):
            states = np.uint64(seq["seed"]) + np.arange(n, dtype=np.uint64) * gamma
        got = [int(v) for v in W.splitmix64(states)]
        assert got == [int(v, 0) for v in seq["outputs"]]


def test_noise_range_and_node_independence():
    shape = (37, 29)
    eps = W.uniform_noise(shape, 5, 1e-3)
    assert eps.shape == shape
    assert np.all(eps >= -1e-3) and np.all(eps < 1e-3)
    assert abs(eps.mean()) < 1e-4 and eps.std() == pytest.approx(1e-3 / math.sqrt(3), rel=0.1)
    # a node's value depends only on (seed, node index): the same index in a
    # longer field gives the same value
    flat = W.uniform_noise((37 * 29 + 100,), 5, 1e-3)
    assert np.array_equal(flat[: 37 * 29], eps.ravel())
    assert not np.array_equal(W.uniform_noise(shape, 6, 1e-3), eps)
    rho = np.full(shape, 0.25)
    assert np.array_equal(W.with_noise(rho, 5, 1e-3), 0.25 * (1 + eps))


def test_target_round_trip():
    rg, rl = 2.1e-3, 0.47
    g, l = rg * 1.004, rl * (1 - 3e-5)
    window = np.exp(np.linspace(math.log(g), math.log(l), S.WINDOW))
    t = S.to_target(g, l, window, rg, rl)
    assert t.size == S.NG + S.NL + S.WINDOW
    assert np.all(t[: S.NG] == t[0]) and t[0] == pytest.approx(S.G_SCALE * math.log(1.004))
    g2, l2, w2 = S.from_target(t, rg, rl)
    assert g2 == pytest.approx(g, rel=1e-14) and l2 == pytest.approx(l, rel=1e-14)
    assert np.allclose(w2, window, rtol=1e-13, atol=0)
    # the shape is clipped to the bulks: the window never leaves [g, l]
    t[S.NG + S.NL] = -0.5
    t[-1] = 1.5
    g3, l3, w3 = S.from_target(t, rg, rl)
    assert w3[0] == pytest.approx(g3, rel=1e-14) and w3[-1] == pytest.approx(l3, rel=1e-14)


def test_extract_recovers_a_window_laid_onto_a_slab():
    """A window linear in the position (so every interpolation is exact) laid
    onto a slab by flat_field is read back by extract at the same positions."""
    ny, g, l = 1024, 0.01, 0.4
    window = g + (l - g) * (S.S - S.S[0]) / (S.S[-1] - S.S[0])
    rho = S.flat_field(4, ny, g, l, window)
    assert rho.shape == (ny, 4) and np.all(rho[:, 0] == rho[:, 3])
    g2, l2, w2 = S.extract(rho[:, 0])
    assert g2 == pytest.approx(g, rel=1e-15) and l2 == pytest.approx(l, rel=1e-15)
    assert np.allclose(w2[1:-1], window[1:-1], rtol=1e-13, atol=0)
    # at the ends the laid profile meets the flat bulk half a node out
    assert abs(w2[0] - window[0]) <= (window[1] - window[0]) / 2


def test_drop_field_profile_is_radial():
    window = np.linspace(0.01, 0.4, S.WINDOW)
    rho = S.drop_field(64, 48, 10.0, 0.01, 0.4, window)
    assert rho[24, 32] == 0.4  # the core r < radius / 2 is the bulk liquid
    assert rho[24, 32 + 7] == pytest.approx(S.profile_at(0.01, 0.4, window, 3.0))
    assert rho[24, 32 + 7] == pytest.approx(rho[24 + 7, 32])  # same distance, same value
    assert rho.min() >= 0.01 and rho.max() <= 0.4


def test_input_scaling_and_sampling():
    r = S.DEFAULT_RANGES
    lo = [v[0] for v in r.values()]
    hi = [v[1] for v in r.values()]
    x = S.scale_inputs([lo[0], hi[0]], [lo[1], hi[1]], [lo[2], hi[2]], r)
    assert x.dtype == np.float32 and np.array_equal(x, [[-1, -1, -1, 0], [1, 1, 1, 0]])
    x = S.scale_inputs([lo[0], hi[0]], [lo[1], hi[1]], [lo[2], hi[2]], r,
                       inv_r=[0.004, 0.016], inv_r_range=(0.004, 0.016))
    assert np.array_equal(x[:, 3], [-1, 1])
    a = S.sample_inputs(500, 3)
    b = S.sample_inputs(500, 3)
    for col, (l0, h0), col_b in zip(a, r.values(), b):
        assert np.all(col >= l0) and np.all(col < h0) and np.array_equal(col, col_b)
    assert not np.array_equal(S.sample_inputs(500, 4)[0], a[0])


class _FakeSim:
    """A run whose probe approaches 1 as 1 + exp(-t / 1000)."""

    def __init__(self):
        self.t = 0

    def step(self, n):
        self.t += n


def test_steps_to_equilibrium_stops_at_the_first_check_within_tolerance():
    probe = lambda s: [1 + math.exp(-s.t / 1000.0)]  # noqa: E731
    # exp(-t/1000) <= 1e-3 first at t = 6908; checks every 500: t = 7000
    assert S.steps_to_equilibrium(_FakeSim(), probe, [1.0], 1e-3, every=500) == 7000
    assert S.steps_to_equilibrium(_FakeSim(), probe, [1.0], 1e-9, every=500,
                                  max_steps=10_000) is None


def test_batch_instances_are_seeded_and_well_formed():
    a = W.batch_instances(64, seed=7)
    assert a == W.batch_instances(64, seed=7)
    assert a != W.batch_instances(64, seed=8)
    assert {d["nx"] for d in a} <= set(W.BATCH_SIDES)
    trs = [d["T_r"] for d in a]
    assert trs[0] == pytest.approx(0.3) and trs[-1] == pytest.approx(0.9)
    assert all(d["k"] == (0.5 if d["T_r"] >= 0.45 else 0.3) for d in a)
    assert {d["kind"] for d in a} == {"drop", "flat"}


def test_extract_drop_on_an_analytic_drop():
    """A tanh drop of known radius and width: the bulks are the two densities
    (the field's own values far from the interface) and the window is the
    profile about the radius, where the midpoint crossing sits."""
    n, R, w, g, l = 256, 64.0, 10.0, 0.02, 0.4
    rho = W.drop(n, n, g, l, R, w)
    eg, el, win = S.extract_drop(rho, R)
    assert eg == pytest.approx(g, rel=2e-3) and el == pytest.approx(l, rel=1e-6)
    exact = 0.5 * (g + l) + 0.5 * (g - l) * np.tanh(2.0 * (-S.S) / w)  # d = R - r
    assert np.abs(win - exact).max() <= 5e-3 * l  # quarter-node bins on the steep flank


def test_settle_step():
    t = list(range(0, 10000, 100))
    v = [(1.0 + np.exp(-ti / 800.0) * np.cos(ti / 50.0), 2.0) for ti in t]
    s = S.settle_step(t, v, (1.0, 2.0), 1e-3, 4)
    # the windowed mean settles once the decaying term is ~1e-3 (t ~ 800 ln 1000)
    assert 4000 <= s <= 6000
    assert S.settle_step(t, v, (1.1, 2.0), 1e-3, 4) is None


def test_drop_radius_for_mass():
    window = 0.2 + 0.18 * np.tanh(S.S / 5.0)
    target = S.drop_field(96, 96, 20.0, 0.02, 0.38, window).sum()
    r = S.drop_radius_for_mass(96, 96, target, 0.02, 0.38, window, 23.0)
    assert r == pytest.approx(20.0, abs=1e-6)
