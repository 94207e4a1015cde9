"""Pins of the oracle's lattice Boltzmann step (Eqs. 1-5, 12, 33), CPU only.

  * the exact-difference forcing of Eq. 5 adds no mass and exactly the momentum F,
    and changes the second moment by rho[(u + F/rho)(u + F/rho) - u u], the
    equilibrium's own change (a Guo-type or first-order forcing does not);
  * at a converged flat interface the fluid velocity v = u + F/(2 rho) of Sec. 2
    vanishes (under 1e-9 after 8000 steps) while the bare moment u = sum e_i f_i / rho does not
    (0.05): this fixes the half-force shift;
  * the equilibrium of Eq. 2 has the textbook moments;
  * a uniform fluid at rest is a fixed point (the compact derivative of a
    constant is exactly zero, so F = 0);
  * a shear wave decays at the BGK viscosity nu = c_s^2 (tau - 1/2) (Sec. 2);
  * mass is conserved to rounding by collision + periodic streaming;
  * the force stage reduces to F = (c_s^2 - k^2 R T) grad(rho) for an ideal-gas
    limit and its sign drives phase separation;
  * where the upper limit caps mu-hat at every node, grad(mu-hat) = 0 and the
    force is exactly c_s^2 D rho: for one Fourier mode of rho, c_s^2 theta(w)
    times its derivative mode (Sec. 5.6 with Eqs. 12, 37-39).
"""
import math

import numpy as np
import pytest

from oracle import OracleSim, forcing_terms, thermo
from paper_1906_09530_gb300 import workloads as W

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
TC, RC = thermo.critical_point()


@pytest.mark.parametrize("rho,ux,uy,Fx,Fy", [(0.4, 0.01, -0.02, 1e-3, 2e-3),
                                             (1e-6, 0.0, 0.05, -1e-8, 3e-9),
                                             (0.2, -0.1, 0.07, 0.0, 0.0)])
def test_forcing_adds_momentum_F(rho, ux, uy, Fx, Fy):
    Fi = forcing_terms(rho, ux, uy, Fx, Fy)
    assert abs(Fi.sum()) < 1e-15 * rho
    assert (EX * Fi).sum() == pytest.approx(Fx, rel=1e-10, abs=1e-18)
    assert (EY * Fi).sum() == pytest.approx(Fy, rel=1e-10, abs=1e-18)


@pytest.mark.parametrize("rho,ux,uy,Fx,Fy", [(0.4, 0.01, -0.02, 1e-3, 2e-3),
                                             (2.0, -0.1, 0.07, -0.05, 0.03)])
def test_forcing_second_moment(rho, ux, uy, Fx, Fy):
    Fi = forcing_terms(rho, ux, uy, Fx, Fy)
    vx, vy = ux + Fx / rho, uy + Fy / rho
    assert (EX * EX * Fi).sum() == pytest.approx(rho * (vx * vx - ux * ux), rel=1e-12)
    assert (EY * EY * Fi).sum() == pytest.approx(rho * (vy * vy - uy * uy), rel=1e-12)
    assert (EX * EY * Fi).sum() == pytest.approx(rho * (vx * vy - ux * uy), rel=1e-12)


def test_flat_equilibrium_is_at_rest_in_the_half_force_velocity():
    tr, k, ny = 0.8, 0.3, 64
    rg, rl = thermo.maxwell(tr)
    sim = OracleSim(4, ny, tr * TC, 0.1, 1.0, k, 6)
    sim.set_fields(W.flat(4, ny, rg, rl, ny / 2, 4.0 / k))
    sim.step(8000)  # measured: |v| 3e-11
    rho, vx, vy = sim.fields()[:3]
    u = (EY[:, None, None] * sim.f).sum(axis=0) / rho
    assert np.abs(vy).max() <= 1e-9 and np.all(vx == 0.0)
    assert np.abs(u).max() >= 0.01


def test_equilibrium_moments():
    sim = OracleSim(8, 8, 0.7 * TC, 0.1, 1.0, 1.0, 4)
    rho = np.full((8, 8), 0.3)
    ux = np.full((8, 8), 0.04)
    uy = np.full((8, 8), -0.03)
    sim.set_fields(rho, ux, uy)
    f = sim.f[:, 0, 0]
    assert f.sum() == pytest.approx(0.3, rel=1e-15)
    assert (EX * f).sum() == pytest.approx(0.3 * 0.04, rel=1e-14)
    assert (EY * f).sum() == pytest.approx(-0.3 * 0.03, rel=1e-14)
    # second moment: sum e_a e_b f = rho (c_s^2 delta_ab + u_a u_b)
    assert (EX * EX * f).sum() == pytest.approx(0.3 * (1 / 3 + 0.04 ** 2), rel=1e-14)
    assert (EX * EY * f).sum() == pytest.approx(0.3 * (0.04 * -0.03), rel=1e-13)


def test_uniform_rest_is_fixed_point():
    sim = OracleSim(16, 12, 0.6 * TC, 0.1, 0.8, 0.5, 6)
    sim.set_fields(np.full((12, 16), 0.25))
    f0 = sim.f.copy()
    _, Fx, Fy = sim.force_stage(np.full((12, 16), 0.25))
    assert np.all(Fx == 0.0) and np.all(Fy == 0.0)
    sim.step(10)
    assert np.allclose(sim.f, f0, rtol=1e-14, atol=0)


def test_shear_wave_viscosity():
    """u_x = U sin(2 pi y / N) at uniform density decays as exp(-nu k^2 t) with
    nu = (tau - 1/2)/3 (Sec. 2, after Eq. 3).  Supercritical T keeps the EOS stable."""
    n, tau, U = 64, 0.8, 1e-5
    sim = OracleSim(4, n, 1.5 * TC, 0.1, tau, 1.0, 6)
    rho, ux, uy = W.shear_wave(4, n, 0.2, U)
    sim.set_fields(rho, ux, uy)
    sim.step(400)
    _, vx, _, _, _, _ = sim.fields()
    y = np.arange(n)
    amp = 2 * np.mean(vx[:, 0] * np.sin(2 * np.pi * y / n))
    nu_meas = -math.log(amp / U) / ((2 * math.pi / n) ** 2 * 400)
    assert nu_meas == pytest.approx((tau - 0.5) / 3, rel=5e-3)


@pytest.mark.parametrize("order", [4, 6])
def test_mass_conserved(order):
    rg, rl = thermo.maxwell(0.6)
    rho = W.with_noise(W.drop(32, 32, rg, rl, 8, 4), 7, 1e-6)
    sim = OracleSim(32, 32, 0.6 * TC, 0.1, 1.0, 0.5, order)
    sim.set_fields(rho)
    m0 = sim.f.sum()
    sim.step(200)
    assert abs(sim.f.sum() - m0) / m0 < 1e-13


def test_force_ideal_gas_limit():
    """In a dilute gas, mu0 ~ R T ln(rho) + const, so with kappa-hat = 0 the force of
    Eq. 12 tends to (c_s^2 - k^2 R T) grad(rho) (Eqs. 21, 33)."""
    n, k = 64, 0.5
    T = 0.4 * TC
    sim = OracleSim(4, n, T, 1e-30, 1.0, k, 6)
    y = np.arange(n)
    rho = 1e-6 * (1 + 1e-3 * np.sin(2 * np.pi * y / n))[:, None] * np.ones((1, 4))
    _, Fx, Fy = sim.force_stage(rho)
    drho = 1e-9 * (2 * np.pi / n) * np.cos(2 * np.pi * y / n)
    expect = (1 / 3 - k * k * T) * drho
    assert np.allclose(Fy[:, 0], expect, rtol=2e-3, atol=1e-3 * np.abs(expect).max())
    assert np.all(Fx == 0.0)


def test_mu_cap_limits_and_keeps_mass():
    """Sec. 5.6: the upper limit clips mu-hat at k^2 mu_max only while t < n_cap and
    leaves the mass untouched."""
    rg, rl = thermo.maxwell(0.6)
    rho = W.drop(24, 24, rg, rl, 6, 4)
    mu_max = -0.3
    capped = OracleSim(24, 24, 0.6 * TC, 0.1, 1.0, 0.5, 6, mu_max=mu_max, mu_cap_steps=5)
    capped.set_fields(rho)
    mu, _, _ = capped.force_stage(capped.fields()[0], t=0)
    assert mu.max() <= 0.25 * mu_max + 1e-15
    free = OracleSim(24, 24, 0.6 * TC, 0.1, 1.0, 0.5, 6)
    free.set_fields(rho)
    mu_free, _, _ = free.force_stage(free.fields()[0], t=0)
    assert mu_free.max() > 0.25 * mu_max
    m0 = capped.f.sum()
    capped.step(10)
    assert abs(capped.f.sum() - m0) / m0 < 1e-13
    mu_late, _, _ = capped.force_stage(capped.fields()[0], t=capped.t)
    assert mu_late.max() > 0.25 * mu_max  # inactive after n_cap


def test_force_where_the_limit_caps_every_node():
    from oracle import cfd_alpha
    n, k, order = 48, 0.5, 6
    T = 0.6 * TC
    y = np.arange(n)[:, None] * np.ones((1, 4))
    w = 2 * np.pi * 3 / n
    rho = 0.45 + 0.02 * np.sin(w * y)  # dense liquid: mu0 far above the limit below
    sim = OracleSim(4, n, T, 0.1, 1.0, k, order, mu_max=-5.0, mu_cap_steps=10)
    mu, Fx, Fy = sim.force_stage(rho, t=0)
    assert np.all(mu == k * k * -5.0)
    a = cfd_alpha(order)
    A, B = 2.0 / 3.0 * (a + 2.0), (4.0 * a - 1.0) / 3.0
    theta = (A * np.sin(w) + B / 2 * np.sin(2 * w)) / (1 + 2 * a * np.cos(w))
    assert np.abs(Fy - 0.02 * theta * np.cos(w * y) / 3).max() <= 1e-15
    assert np.all(Fx == 0.0)


def test_threads_do_not_change_the_bits():
    """The C oracle shares its loops over lines and nodes among threads when
    built with OpenMP; every line and node is computed as with one thread, so a
    run gives the same bits with 1 and with 4 threads (periodic and walled)."""
    from oracle import sim as S
    from oracle import thermo as T
    from paper_1906_09530_gb300 import workloads as W
    Tc, _ = T.critical_point()
    rg, rl = T.maxwell(0.6)
    rho = W.with_noise(W.drop(48, 40, rg, rl, 10.0, 4.0), 7, 1e-4)
    out = []
    try:
        for n in (1, 4):
            S.set_threads(n)
            for walls in (False, True):
                o = S.OracleSim(48, 40, 0.6 * Tc, 0.1, 0.9, 0.5, 6, walls_y=walls)
                o.set_fields(rho)
                o.step(30)
                out.append(o.f.copy())
    finally:
        S.set_threads(1)
    assert np.array_equal(out[0], out[2]) and np.array_equal(out[1], out[3])
