"""Pins of the oracle's walls (Sec. 5.5: periodic in x, solid top and bottom).

Populations: halfway bounce-back, so the no-slip wall lies half a node outside
the first and last rows.  Derivatives in y: every field is extended evenly
about both walls, so the first ghost takes its fluid neighbour's value (the
paper's wall rule for the chemical potential) and each y-line becomes periodic
with period 2 ny.

  * the y-derivative of cos(m pi (y + 1/2)/ny), even about both walls, is the
    compact scheme's modified wavenumber times -sin(...), exactly (Eqs. 37-39);
    a ghost reflected about the wrong point, or an odd extension, fails;
  * the second y-derivative of the force stage (the scheme applied twice along
    the extended density line) of that mode is -theta^2 times it, exactly, and
    mu-hat of a small such ripple is k^2 mu0(rho) + kappa theta^2 times the
    ripple; re-extending the intermediate first derivative evenly fails;
  * the no-slip shear mode u_x = U sin(pi (y + 1/2)/ny) between the walls decays
    as exp(-nu (pi/ny)^2 t), nu = (tau - 1/2)/3: this fixes the wall position;
  * with the walls moving along x at U_b and U_t (Ladd's moving-wall rule),
    steady Couette flow is u_x = U_b + (U_t - U_b)(y + 1/2)/ny to rounding,
    for any tau: this fixes the sign and the weight of the wall momentum;
  * with the MRT collision (Eq. 4) the same Couette flow is linear up to a
    compressibility term of third order in the wall speed (its deviation falls
    eightfold when the speeds halve; 6e-8 at U_t - U_b = 0.04), where a wrong
    wall momentum would leave a first-order error;
  * bounce-back conserves mass to rounding, moving walls too;
  * the even extension is a neutral wall: a drop that starts as a cap meeting
    the wall at 124 degrees relaxes to a half-disk, a contact angle of 90
    degrees (measured 89.4 after 1000 steps, from tan(theta/2) = h/b with the
    interpolated height h and base half-width b);
  * without walls the same calls reduce to the periodic ones.
"""
import math

import numpy as np
import pytest

from oracle import OracleSim, cfd_alpha, thermo
from paper_1906_09530_gb300 import workloads as W

TC, _ = thermo.critical_point()


def theta(order, w):
    a = cfd_alpha(order)
    A = 2.0 / 3.0 * (a + 2.0)
    B = (4.0 * a - 1.0) / 3.0
    return (A * math.sin(w) + B / 2 * math.sin(2 * w)) / (1 + 2 * a * math.cos(w))


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("m", [1, 3, 7])
def test_even_extension_derivative(order, m):
    nx, ny = 3, 24
    s = OracleSim(nx, ny, 0.7 * TC, 0.1, 1.0, 0.5, order, walls_y=True)
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    w = m * math.pi / ny
    u = np.cos(w * (y + 0.5))
    d = s.cfd_field(u, 1)
    assert np.abs(d + theta(order, w) * np.sin(w * (y + 0.5))).max() <= 1e-13
    # x stays periodic
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    ux = np.sin(2 * math.pi * x / nx)
    assert np.abs(s.cfd_field(ux, 0) - theta(order, 2 * math.pi / nx) *
                  np.cos(2 * math.pi * x / nx)).max() <= 1e-13


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("m", [1, 4, 9])
def test_second_derivative_along_extended_line(order, m):
    nx, ny = 3, 24
    s = OracleSim(nx, ny, 0.7 * TC, 0.1, 1.0, 0.5, order, walls_y=True)
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    w = m * math.pi / ny
    u = np.cos(w * (y + 0.5))
    assert np.abs(s.cfd_field(u, 2) + theta(order, w) ** 2 * u).max() <= 1e-13


@pytest.mark.parametrize("order", [4, 6])
def test_mu_hat_of_a_wall_ripple(order):
    nx, ny, T_r, kappa, k, eps = 4, 30, 0.8, 0.1, 0.5, 1e-3
    T = T_r * TC
    s = OracleSim(nx, ny, T, kappa, 1.0, k, order, walls_y=True)
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    w = 2 * math.pi / ny
    ripple = eps * np.cos(w * (y + 0.5))
    rho = 0.3 + ripple
    mu, _, _ = s.force_stage(rho)
    want = k * k * thermo.mu0(rho, T) + kappa * theta(order, w) ** 2 * ripple
    assert np.abs(mu - want).max() <= 1e-13


def test_channel_shear_mode_decay():
    nx, ny, tau, U = 4, 32, 1.0, 1e-5
    s = OracleSim(nx, ny, 1.5 * TC, 0.1, tau, 1.0, 6, walls_y=True)
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    ux = U * np.sin(math.pi * (y + 0.5) / ny)
    s.set_fields(np.full((ny, nx), 0.2), ux, np.zeros_like(ux))
    s.step(2000)
    vx = s.fields()[1]
    prof = np.sin(math.pi * (np.arange(ny) + 0.5) / ny)
    amp = (vx[:, 0] @ prof) / (prof @ prof)
    nu = -math.log(amp / U) / ((math.pi / ny) ** 2 * 2000)
    assert nu == pytest.approx((tau - 0.5) / 3, rel=1e-2)


@pytest.mark.parametrize("tau", [0.7, 1.0, 1.6])
def test_couette_flow_between_moving_walls(tau):
    nx, ny, ub, ut = 4, 16, -0.01, 0.03
    s = OracleSim(nx, ny, 1.5 * TC, 0.1, tau, 1.0, 6, walls_y=True, wall_ux=(ub, ut))
    s.set_fields(np.full((ny, nx), 0.2))
    s.step(int(6 * ny * ny / ((tau - 0.5) / 3)))  # many viscous times
    rho, vx, vy, *_ = s.fields()
    y = np.arange(ny)[:, None]
    assert np.abs(vx - (ub + (ut - ub) * (y + 0.5) / ny)).max() <= 1e-12
    assert np.abs(vy).max() <= 1e-13
    assert np.abs(rho - 0.2).max() <= 1e-12


def test_couette_flow_with_mrt_is_linear_to_third_order():
    from oracle import sim as S
    nx, ny, tau = 4, 16, 1.0
    dev = []
    for scale in (1.0, 0.5):
        ub, ut = -0.01 * scale, 0.03 * scale
        s = OracleSim(nx, ny, 1.5 * TC, 0.1, tau, 1.0, 6, walls_y=True, wall_ux=(ub, ut),
                      mrt=S.PAPER_MRT)
        s.set_fields(np.full((ny, nx), 0.2))
        s.step(int(6 * ny * ny / ((tau - 0.5) / 3)))
        vx = s.fields()[1]
        y = np.arange(ny)[:, None]
        dev.append(np.abs(vx - (ub + (ut - ub) * (y + 0.5) / ny)).max())
    assert dev[0] <= 1e-7
    assert 7.0 <= dev[0] / dev[1] <= 9.0, dev


def test_mass_conserved_with_moving_walls():
    rg, rl = thermo.maxwell(0.6)
    rho = W.with_noise(W.drop(40, 32, rg, rl, 8, 4, center=(20, 10)), 7, 1e-6)
    s = OracleSim(40, 32, 0.6 * TC, 0.1, 1.0, 0.5, 6, walls_y=True, wall_ux=(0.05, 0.05))
    s.set_fields(rho, np.full_like(rho, 0.05), np.full_like(rho, -0.02))
    m0 = s.f.sum()
    s.step(200)
    assert abs(s.f.sum() - m0) / m0 < 1e-13


def test_mass_conserved_with_walls():
    rg, rl = thermo.maxwell(0.6)
    rho = W.with_noise(W.drop(40, 32, rg, rl, 8, 4, center=(20, 10)), 7, 1e-6)
    s = OracleSim(40, 32, 0.6 * TC, 0.1, 1.0, 0.5, 6, walls_y=True)
    s.set_fields(rho, np.zeros_like(rho), np.full_like(rho, -0.02))
    m0 = s.f.sum()
    s.step(200)
    assert abs(s.f.sum() - m0) / m0 < 1e-13
    assert np.isfinite(s.f).all()


def test_no_walls_is_periodic():
    rg, rl = thermo.maxwell(0.7)
    rho = W.with_noise(W.drop(24, 20, rg, rl, 6, 4), 3, 1e-5)
    a = OracleSim(24, 20, 0.7 * TC, 0.1, 1.0, 0.5, 6)
    b = OracleSim(24, 20, 0.7 * TC, 0.1, 1.0, 0.5, 6, walls_y=False)
    a.set_fields(rho)
    b.set_fields(rho)
    a.step(20)
    b.step(20)
    assert np.array_equal(a.f, b.f)


def test_neutral_wall_relaxes_a_drop_to_a_right_contact_angle():
    tr, k, nx, ny, R = 0.7, 0.5, 80, 48, 14.0
    rg, rl = thermo.maxwell(tr)
    mid = 0.5 * (rg + rl)

    def cap_angle(r):
        """tan(theta/2) = h / b for a circular cap: b the base half-width on
        the first row, h the height of the top crossing above the wall (which
        lies half a node below the first row), both by linear interpolation."""
        row, c = r[0], nx // 2
        i = c
        while row[i + 1] > mid:
            i += 1
        xr = i + (row[i] - mid) / (row[i] - row[i + 1])
        i = c
        while row[i - 1] > mid:
            i -= 1
        xl = i - (row[i] - mid) / (row[i] - row[i - 1])
        col, j = r[:, c], 0
        while col[j + 1] > mid:
            j += 1
        h = j + (col[j] - mid) / (col[j] - col[j + 1]) + 0.5
        return math.degrees(2 * math.atan(h / ((xr - xl) / 2)))

    rho = W.drop(nx, ny, rg, rl, R, 4.0, center=(nx / 2, 7.5))  # centre 8 above the wall
    assert cap_angle(rho) > 120
    s = OracleSim(nx, ny, tr * TC, 0.1, 1.0, k, 6, walls_y=True)
    s.set_fields(rho)
    s.step(1000)
    assert abs(cap_angle(s.fields()[0]) - 90.0) <= 1.5
