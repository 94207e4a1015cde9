"""Pins of the oracle's direct equilibrium solver (oracle/equilibrium.py), and
what it finds about the method's flat coexistence (Sec. 5.1, Fig. 4).

The solver is a second, independent restatement of the time step (numpy, on
the six populations of a slab uniform in x).  It is pinned against the C
oracle, which the other oracle tests pin against the paper:
  * its compact-derivative matrix is the C oracle's periodic line solve;
  * its time step is the C oracle's step, population by population;
  * its fixed point is where the C oracle's time stepping ends;
  * the fixed point does not depend on tau, as Sec. 5.1 states of its results.

What it finds, from the stored study (tests/golden/flat_coexistence.json,
written by tests/golden/make_flat_coexistence.py from oracle/ only; one entry is
recomputed here to tie the file to the code):
  * the liquid sits on Maxwell's density at every temperature (within 1e-4);
  * the gas sits above Maxwell's density by an offset that falls as k^2: the
    measured order is 1.9-2.3 between k 0.1 and 0.05 at every temperature from
    T_r 0.6 down to 0.16;
  * at the paper's k = 0.1 that offset grows as the temperature falls:
    0.027 decade at T_r 0.4, 0.12 at 0.3, 0.65 at 0.2 and 1.7 decades at 0.16
    (where Fig. 4d shows the CS gas on Maxwell's curve down to a density ratio
    above 1e14); at k = 0.05 it is 0.29 decade at T_r 0.2 and 1.0 at 0.16;
  * below T_r ~ 0.25 the dilute gas is 1e9 and more times below the liquid, and
    the solver's Newton step leaves it unresolved; those entries are finished
    by the C oracle's time stepping to a relative residual below 1e-12 (and the
    GPU's FP64 path, run long from a tanh start, ends on the same gas to 1e-9);
  * the known gap: at k = 0.5 (the 1024x1024 drop workload's) the gas is 0.1 to
    1.6 above Maxwell, not within 1e-3 (xfail, strict).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import equilibrium as E
from oracle import sim
from oracle.eos import Eos


def gold():
    with open(os.path.join(os.path.dirname(__file__), "golden", "flat_coexistence.json")) as fh:
        return json.load(fh)


def test_cfd_matrix_is_the_c_oracle_line_solve():
    rng = np.random.default_rng(1)
    for n, order in ((50, 6), (37, 4), (8, 6)):
        u = rng.standard_normal(n)
        d = E.cfd_matrix(n, order) @ u
        assert np.abs(d - sim.cfd_line(u, sim.cfd_alpha(order))).max() <= 1e-13


def test_step_is_the_c_oracle_step():
    T_r, kap, tau, k, n = 0.6, 0.1, 0.8, 0.5, 64
    f, _ = E.slab_start(n, T_r, kap, tau, k, steps=300)
    slab = E.FlatSlab(n, T_r, kap, tau, k)
    Tc, _ = Eos("cs").critical_point()
    o = sim.OracleSim(8, n, T_r * Tc, kap, tau, k, 6)
    o.set_populations(f.copy(), 300)
    o.step(1)
    assert np.abs(slab.step(slab.from_populations(f)) - slab.from_populations(o.f)).max() <= 1e-15


def test_fixed_point_is_where_time_stepping_ends():
    T_r, kap, tau, k, n = 0.7, 0.1, 1.0, 0.5, 32
    r = E.flat_equilibrium(n, T_r, kap, tau, k, steps=2000)
    assert r["residual"] < 1e-13
    Tc, _ = Eos("cs").critical_point()
    f0, _ = E.slab_start(n, T_r, kap, tau, k, steps=0)
    o = sim.OracleSim(8, n, T_r * Tc, kap, tau, k, 6)
    o.set_populations(f0, 0)
    o.step(10000)
    rho = o.fields()[0]
    assert np.abs(rho[:, 0] / r["rho"] - 1).max() <= 1e-11
    assert np.abs(rho - rho[:, :1]).max() == 0.0  # uniform in x, as the reduction assumes
    assert np.abs(r["v"]).max() < 1e-12  # at rest: v = u + F/(2 rho) = 0


def test_fixed_point_does_not_depend_on_tau():
    """Sec. 5.1: the coexistence results do not depend on the relaxation time."""
    rho = [E.flat_equilibrium(64, 0.6, 0.1, tau, 0.5, steps=3000)["rho"] for tau in (0.8, 1.5)]
    assert np.abs(rho[0] / rho[1] - 1).max() <= 1e-10


def test_stored_study_is_what_the_solver_gives():
    e = next(x for x in gold()["k_series"] if x["T_r"] == 0.6 and x["k"] == 0.4)
    r = E.flat_equilibrium(e["height"], 0.6, 0.1, 1.0, 0.4, steps=20000)
    assert r["rho_g"] == pytest.approx(e["rho_g"], rel=1e-9)
    assert r["rho_l"] == pytest.approx(e["rho_l"], rel=1e-12)


def test_liquid_on_maxwell_at_every_temperature():
    for e in gold()["curve_k0.1"] + gold()["k_series"]:
        assert abs(e["liq_offset"]) <= (1e-4 if e["k"] <= 0.2 else 2e-4), e
        assert e["relative_residual"] < 1e-10, e  # every population, gas included


def test_gas_offset_falls_as_k_squared():
    """The gas offset over Maxwell is a discretisation error of the method: it
    vanishes at second order in k at fixed temperature (height 40/k, so the
    domain holds the same interface in the momentum space)."""
    series = {}
    for e in gold()["k_series"]:
        series.setdefault(e["T_r"], {})[e["k"]] = e["gas_offset"]
    for T_r, s in series.items():
        ks = sorted(s)
        assert all(s[k] > 0 for k in ks), (T_r, s)
        # order between the two finest spacings of each temperature
        k1, k2 = ks[0], ks[1]
        order = math.log(s[k2] / s[k1]) / math.log(k2 / k1)
        assert 1.8 <= order <= 2.4, (T_r, order, s)


def test_gas_offset_at_the_paper_k_grows_as_temperature_falls():
    """At k = 0.1 the offset is below 1e-3 relative only above T_r ~ 0.6 and
    reaches decades at the paper's lowest temperatures (Fig. 4d plots the CS
    gas branch down to a density ratio above 1e14)."""
    curve = sorted(gold()["curve_k0.1"], key=lambda e: -e["T_r"])
    offs = [e["gas_offset"] for e in curve]
    assert all(b > a for a, b in zip(offs, offs[1:])), offs
    dec = {e["T_r"]: e["gas_offset_decades"] for e in curve}
    assert dec[0.8] < 1e-3 / math.log(10)
    assert 0.1 < dec[0.3] < 0.15
    assert 0.6 < dec[0.2] < 0.7
    assert 1.5 < dec[0.16] < 1.8


@pytest.mark.xfail(strict=True, reason="known gap: at k = 0.5 (the 1024x1024 drop workload's k) the flat gas "
                   "density is above Maxwell by 1.2e-1 (T_r 0.6), 5.2e-1 (0.5) and 1.6 "
                   "(0.45); the offset falls as k^2, so 1e-3 needs k of about 0.05 at T_r 0.6")
@pytest.mark.parametrize("T_r", [0.6, 0.5, 0.45])
def test_gas_within_1e3_of_maxwell_at_k_half(T_r):
    r = E.flat_equilibrium(64, T_r, 0.1, 1.0, 0.5, steps=4000)
    assert abs(r["liq_offset"]) <= 1e-3
    assert abs(r["gas_offset"]) <= 1e-3, r["gas_offset"]


# ---- the audit of other readings (Eqs. 5, 12, 26; the step order) ----------

def test_mesh_scaled_sound_speed_leaves_no_coexistence():
    """Taking c_s^2 in Eq. 12 as the mesh-space k^2 c_s^2 of Eq. 26 leaves part of
    the lattice's own ideal pressure c_s^2 rho uncancelled: at rest the momentum
    balance becomes grad[(1 - k^2) rho / 3 + k^2 p0(rho)] = 0 in a bulk, an
    effective pressure with no van der Waals loop at the paper's k, so no two
    phases can coexist at all."""
    eos = Eos("cs")
    Tc, _ = eos.critical_point()
    rho = np.linspace(1e-6, 0.9 * eos.rho_max, 20000)
    for k in (0.1, 0.5):
        for T_r in (0.3, 0.6):
            p_eff = (1 - k * k) * rho / 3 + k * k * eos.p0(rho, T_r * Tc)
            assert np.all(np.diff(p_eff) > 0), (k, T_r)
    # while the printed reading's k^2 p0 has the loop that makes two phases
    assert np.any(np.diff(eos.p0(rho, 0.6 * Tc)) < 0)


def test_collision_towards_v_is_unstable():
    """Relaxing towards f^eq(rho, v) with v = u + F/(2 rho): the uniform gas at
    rest already has a growing mode (largest Jacobian eigenvalue above 1)."""
    for reading, unstable in (("printed", False), ("collide_to_v", True)):
        slab = E.FlatSlab(32, 0.6, 0.1, 1.0, 0.5, reading=reading)
        rg, _ = slab.eos.maxwell(0.6)
        g = slab.feq(np.full(32, rg), np.zeros(32))
        lam = np.abs(np.linalg.eigvals(slab.jacobian(g) + np.eye(6 * 32))).max()
        assert (lam > 1.1) == unstable, (reading, lam)


def test_forcing_about_v_moves_the_gas_further():
    """The increment of Eq. 5 taken about v instead of u: an equilibrium exists
    but its gas is ten times further from Maxwell than the printed reading's."""
    printed = E.flat_equilibrium(64, 0.6, 0.1, 1.0, 0.5, steps=3000)
    at_v = E.flat_equilibrium(64, 0.6, 0.1, 1.0, 0.5, steps=3000, reading="forcing_at_v")
    assert at_v["residual"] < 1e-12
    assert at_v["gas_offset"] > 10 * printed["gas_offset"] > 1.0


def test_central_ideal_term_diverges():
    """The c_s^2 grad rho of Eq. 12 by the central difference, the rest as
    printed: the run from a slab leaves the finite numbers within 4000 steps.
    With the compact scheme for both terms of Eq. 12 the lattice's own pressure
    gradient and the force balance at leading order (an exact derivative), which
    is what holds the printed reading's coexistence on Maxwell at leading order."""
    slab = E.FlatSlab(64, 0.6, 0.1, 1.0, 0.5, reading="ideal_central")
    f, _ = E.slab_start(64, 0.6, 0.1, 1.0, 0.5, steps=0)
    g = slab.from_populations(f)
    with np.errstate(all="ignore"):
        for _ in range(4000):
            g = slab.step(g)
            if not np.all(np.isfinite(g)) or slab.moments(g)[0].min() <= 0:
                break
    assert not (np.all(np.isfinite(g)) and slab.moments(g)[0].min() > 0)


def test_step_order_does_not_move_the_fixed_point():
    """Sampling the density after the streaming or after the collision gives the
    same field (the collision conserves mass), and the force depends on the
    density only: a run that takes F from either sees the same force, so every
    ordering of the same step has the same equilibrium densities.  Checked: the
    post-collision state of the fixed point has the fixed point's density."""
    slab = E.FlatSlab(32, 0.7, 0.1, 0.8, 0.5)
    r = E.flat_equilibrium(32, 0.7, 0.1, 0.8, 0.5, steps=2000)
    g = r["g"]
    rho, j = slab.moments(g)
    _, F = slab.force(rho)
    u = j / rho
    feq = slab.feq(rho, u)
    post = g - (g - feq) / slab.tau + slab.feq(rho, u + F / rho) - feq
    assert np.abs(slab.moments(post)[0] / rho - 1).max() <= 1e-14
