"""Pins of the oracle's MRT collision (Eq. 4): f* = f - M^-1 S M (f - f^eq) + F_i,
M the standard D2Q9 moment basis (rows rho, e, epsilon, j_x, q_x, j_y, q_y, p_xx,
p_xy), S = diag(0, s_e, s_eps, 0, s_q, 0, s_q, s_v, s_v), s_v = 1/tau.

  * M applied to f^eq (Eq. 2) gives the known equilibrium moments of that basis,
    so a wrong row or sign in M fails;
  * with every rate equal to 1/tau the MRT collision is the BGK collision of
    Eq. 1 (S = I/tau and M^-1 M = I);
  * mass is conserved to rounding (the rates of rho and j are 0);
  * a shear wave decays at nu = (1/s_v - 1/2)/3, whatever s_e, s_eps and s_q are;
  * a sound wave decays at Gamma = q^2 (nu + zeta)/2 with the bulk viscosity
    zeta = (1/s_e - 1/2)/3, set by the energy mode's rate alone: changing s_eps
    or s_q leaves it unchanged, so s_e sits on the row of e (a swap with s_eps
    fails).
"""
import math

import numpy as np
import pytest

from oracle import OracleSim, sim, thermo
from paper_1906_09530_gb300 import workloads as W

TC, _ = thermo.critical_point()
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def feq(rho, ux, uy):
    eu = EX * ux + EY * uy
    return W9 * rho * (1 + 3 * eu + 4.5 * eu**2 - 1.5 * (ux * ux + uy * uy))


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (0.37, 0.05, -0.02), (2.5, -0.1, 0.07)])
def test_basis_on_equilibrium(rho, ux, uy):
    M, Mi = sim.mrt_matrices()
    m = M @ feq(rho, ux, uy)
    u2 = ux * ux + uy * uy
    want = [rho, rho * (-2 + 3 * u2), rho * (1 - 3 * u2), rho * ux, -rho * ux, rho * uy,
            -rho * uy, rho * (ux * ux - uy * uy), rho * ux * uy]
    assert np.allclose(m, want, rtol=1e-14, atol=1e-15)
    assert np.allclose(M @ Mi, np.eye(9), atol=1e-15)


def test_equal_rates_reduce_to_bgk():
    rg, rl = thermo.maxwell(0.7)
    rho = W.with_noise(W.drop(32, 28, rg, rl, 8, 4), 5, 1e-5)
    tau = 0.8
    a = OracleSim(32, 28, 0.7 * TC, 0.1, tau, 0.5, 6)
    b = OracleSim(32, 28, 0.7 * TC, 0.1, tau, 0.5, 6, mrt=(1 / tau, 1 / tau, 1 / tau))
    a.set_fields(rho)
    b.set_fields(rho)
    a.step(60)
    b.step(60)
    assert np.abs(a.f - b.f).max() <= 1e-14 * np.abs(a.f).max()


def test_mass_conserved():
    rg, rl = thermo.maxwell(0.6)
    rho = W.with_noise(W.drop(32, 32, rg, rl, 8, 4), 7, 1e-6)
    s = OracleSim(32, 32, 0.6 * TC, 0.1, 1.0, 0.5, 6, mrt=sim.PAPER_MRT)
    s.set_fields(rho)
    m0 = s.f.sum()
    s.step(200)
    assert abs(s.f.sum() - m0) / m0 < 1e-13


@pytest.mark.parametrize("rates", [sim.PAPER_MRT, (1.2, 1.0, 1.5)])
def test_shear_wave_viscosity(rates):
    n, tau, U = 64, 0.8, 1e-5
    s = OracleSim(4, n, 1.5 * TC, 0.1, tau, 1.0, 6, mrt=rates)
    rho, ux, uy = W.shear_wave(4, n, 0.2, U)
    s.set_fields(rho, ux, uy)
    s.step(400)
    _, vx, _, _, _, _ = s.fields()
    y = np.arange(n)
    amp = 2 * np.mean(vx[:, 0] * np.sin(2 * np.pi * y / n))
    nu = -math.log(amp / U) / ((2 * math.pi / n) ** 2 * 400)
    assert nu == pytest.approx((tau - 0.5) / 3, rel=5e-3)


def _sound_damping(rates, n=64, steps=1500):
    """Decay rate of the envelope of a small standing sound wave (nearly ideal
    fluid: T = 1.5 T_c, kappa-hat ~ 0, k = 1), from its peaks."""
    o = OracleSim(n, 4, 1.5 * TC, 1e-30, 1.0, 1.0, 6, mrt=rates)
    x = np.arange(n)[None, :] * np.ones((4, 1))
    o.set_fields(0.2 * (1 + 1e-4 * np.cos(2 * np.pi * x / n)))
    c = np.cos(2 * np.pi * np.arange(n) / n)
    amp = []
    for _ in range(steps // 5):
        o.step(5)
        r = o.fields()[0][0]
        amp.append(abs((r - r.mean()) @ c) / (n / 2))
    amp, t = np.array(amp), 5.0 * np.arange(1, len(amp) + 1)
    pk = [i for i in range(1, len(amp) - 1) if amp[i] >= amp[i - 1] and amp[i] >= amp[i + 1]]
    return -np.polyfit(t[pk], np.log(amp[pk]), 1)[0], (2 * np.pi / n) ** 2


def test_sound_wave_bulk_viscosity():
    nu = (1.0 - 0.5) / 3  # tau = 1
    g = {}
    for name, rates in (("paper", (1.64, 1.54, 1.9)), ("se1", (1.0, 1.54, 1.9)),
                        ("seps", (1.64, 1.0, 1.9)), ("sq", (1.64, 1.54, 1.2))):
        g[name], q2 = _sound_damping(rates)
    for name, se in (("paper", 1.64), ("se1", 1.0)):
        zeta = 2 * g[name] / q2 - nu
        assert zeta == pytest.approx((1 / se - 0.5) / 3, rel=0.02), (name, zeta)
    assert g["seps"] == pytest.approx(g["paper"], rel=1e-3)
    assert g["sq"] == pytest.approx(g["paper"], rel=1e-3)
