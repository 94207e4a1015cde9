"""The learned warm start (paper_1906_09530_gb300.surrogate): the network is
trained by the library's own kernels (test_gpu_mlp.py checks their gradients
against the oracle) on equilibrium flat interfaces produced by the batched
path, and this test shows what it gains over the method without it.

Inputs vary T_r over 0.36-0.48 at kappa-hat = 0.1, k = 0.2, where the method's
gas branch settles 10-30% above Maxwell (the discrete scheme's offset).  A tanh
start between the Maxwell densities must relax that offset by mass diffusion
through the gas, which is slow in a tall domain.  The warm start begins within
a few tenths of a percent of it.
"""
import numpy as np
import pytest

from paper_1906_09530_gb300 import workloads as W

pytestmark = pytest.mark.gpu
RANGES = {"T_r": (0.36, 0.48), "kappa": (0.1, 0.1), "k": (0.2, 0.2)}


@pytest.fixture(scope="module")
def trained(cuda):
    from paper_1906_09530_gb300 import surrogate as SG
    n = 96
    T = np.linspace(*RANGES["T_r"], n)
    K, k = np.full(n, 0.1), np.full(n, 0.2)
    G, L, P = SG.equilibrium_profiles(T, K, k, steps=150_000)
    s = SG.Surrogate(seed=3, ranges=RANGES)
    loss = s.fit(T, K, k, G, L, P, epochs=3000, lr=2e-3, batch=96)
    yield s, loss
    s.close()


def _bulk(sim, ny):
    r = sim.fields()[0][:, 0]
    return (np.r_[r[: ny // 10], r[-ny // 10:]].mean(),
            r[ny // 2 - ny // 10: ny // 2 + ny // 10].mean())


def test_prediction_matches_held_out_equilibrium(trained):
    from paper_1906_09530_gb300 import surrogate as SG
    s, loss = trained
    assert loss < 1e-5
    T = np.array([0.39, 0.42, 0.45])
    G, L, P = SG.equilibrium_profiles(T, np.full(3, 0.1), np.full(3, 0.2), steps=150_000)
    g, l, w = s.predict(T, 0.1 * np.ones(3), 0.2 * np.ones(3))
    # the gas offset over Maxwell is 10-30% here; the seeded fit predicts it to
    # 0.2-0.5% (the spread between network initialisations), the bound is 1%
    assert np.abs(g / G - 1).max() <= 1e-2
    assert np.abs(l / L - 1).max() <= 1e-4
    # the interface shape, compared in log density across the window
    span = np.log(L) - np.log(G)
    assert (np.abs(np.log(w) - np.log(P)) / span[:, None]).max() <= 2e-2


def test_warm_start_reaches_equilibrium_sooner(trained):
    """Tall slab (8 x 1536) at T_r = 0.42: steps until both bulk densities are
    within 1e-3 of the equilibrium of a long run, from the tanh start and from
    the warm start.  Measured: 54 000 and 0."""
    from paper_1906_09530_gb300 import Simulation, lbm_maxwell
    from paper_1906_09530_gb300 import surrogate as SG
    s, _ = trained
    T, K, k, ny = 0.42, 0.1, 0.2, 1536
    rg, rl = lbm_maxwell(T)
    ref = Simulation(8, ny, T, K, 1.0, k, fd_order=6, precision="mixed")
    ref.set_fields(W.flat(8, ny, rg, rl, ny / 2, 4.0 / k))
    ref.step(1_000_000)
    eq = _bulk(ref, ny)
    ref.close()
    g, l, w = s.predict([T], [K], [k])
    steps = {}
    for name, field in (("tanh", W.flat(8, ny, rg, rl, ny / 2, 4.0 / k)),
                        ("warm", SG.flat_field(8, ny, g[0], l[0], w[0]))):
        sim = Simulation(8, ny, T, K, 1.0, k, fd_order=6, precision="mixed")
        sim.set_fields(field)
        steps[name] = SG.steps_to_equilibrium(sim, lambda x: _bulk(x, ny), eq, 1e-3,
                                              every=2000, max_steps=400_000)
        sim.close()
    assert steps["tanh"] is not None and steps["tanh"] >= 20_000
    assert steps["warm"] is not None and steps["warm"] <= steps["tanh"] / 3
