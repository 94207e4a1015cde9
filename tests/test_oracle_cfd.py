"""Pins of the oracle's compact finite differences (Eqs. 37-39), CPU only.

  * exactness on every discrete Fourier mode against the closed-form modified
    wavenumber of the scheme;
  * brute force: the dense cyclic system solved by LU for small n;
  * the formal order (4 for alpha = 1/4, 6 for alpha = 1/3) on sine fields;
  * the printed Eq. 39 coefficients.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import cfd_alpha, cfd_line

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def coeffs(alpha):
    return 2.0 / 3.0 * (alpha + 2.0), (4.0 * alpha - 1.0) / 3.0  # Eq. 38


def test_eq39_coefficients():
    g = GOLD["cfm_sixth"]
    a, b = coeffs(cfd_alpha(6))
    assert cfd_alpha(6) == pytest.approx(g["alpha"]) and a == pytest.approx(g["a"])
    assert b == pytest.approx(g["b"])
    a4, b4 = coeffs(cfd_alpha(4))
    assert (a4, b4) == (1.5, 0.0)


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("n", [8, 17, 64])
def test_modified_wavenumber_exact(order, n):
    """For u_j = sin(theta j + phi) the periodic scheme returns exactly
    w'(theta) cos(theta j + phi) with
    w'(theta) = [a sin(theta) + (b/2) sin(2 theta)] / (1 + 2 alpha cos(theta))."""
    alpha = cfd_alpha(order)
    a, b = coeffs(alpha)
    j = np.arange(n)
    for m in range(0, n // 2 + 1):
        th = 2 * math.pi * m / n
        u = np.sin(th * j + 0.3)
        wp = (a * math.sin(th) + 0.5 * b * math.sin(2 * th)) / (1 + 2 * alpha * math.cos(th))
        assert np.allclose(cfd_line(u, alpha), wp * np.cos(th * j + 0.3), rtol=0, atol=1e-13)


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("n", [5, 8, 13, 32])
def test_dense_bruteforce(order, n):
    alpha = cfd_alpha(order)
    a, b = coeffs(alpha)
    A = np.eye(n)
    B = np.zeros((n, n))
    for i in range(n):
        A[i, (i - 1) % n] += alpha
        A[i, (i + 1) % n] += alpha
        B[i, (i + 1) % n] += a / 2
        B[i, (i - 1) % n] -= a / 2
        B[i, (i + 2) % n] += b / 4
        B[i, (i - 2) % n] -= b / 4
    rng = np.random.default_rng(n)
    u = rng.standard_normal(n)
    ref = np.linalg.solve(A, B @ u)
    assert np.allclose(cfd_line(u, alpha), ref, rtol=0, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("order,ratio", [(4, 16.0), (6, 64.0)])
def test_formal_order(order, ratio):
    alpha = cfd_alpha(order)
    errs = []
    for n in (16, 32, 64):
        x = np.arange(n) * (2 * math.pi / n)
        d = cfd_line(np.sin(x), alpha, h=2 * math.pi / n)
        errs.append(np.abs(d - np.cos(x)).max())
    assert errs[0] / errs[1] == pytest.approx(ratio, rel=0.05)
    assert errs[1] / errs[2] == pytest.approx(ratio, rel=0.05)


def test_constant_gives_zero_exactly():
    for order in (4, 6):
        assert np.all(cfd_line(np.full(20, 0.37), cfd_alpha(order)) == 0.0)


def test_sixth_beats_second_order_cdm_on_profile():
    """Sec. 4.3 / Fig. 2: on a smooth but steep interface profile the compact
    scheme is far more accurate than the second-order central difference (Eq. 34)."""
    n = 64
    x = np.arange(n)
    w = 2.0
    u = np.tanh((x - n / 4) / w) - np.tanh((x - 3 * n / 4) / w)
    exact = (1 / np.cosh((x - n / 4) / w) ** 2 - 1 / np.cosh((x - 3 * n / 4) / w) ** 2) / w
    cdm2 = (np.roll(u, -1) - np.roll(u, 1)) / 2
    e_cfm = np.abs(cfd_line(u, cfd_alpha(6)) - exact).max()
    e_cdm = np.abs(cdm2 - exact).max()
    assert e_cfm < e_cdm / 20
