"""Pins of the oracle's equation of state and thermodynamics (CPU only).

Each test ties the oracle to something outside itself: the textbook virial
series of the Carnahan-Starling fluid, the Gibbs-Duhem identity between the
independently printed Eqs. 20 and 21, the definition of the critical point, the
equal-area rule of the Maxwell construction, and constants the paper prints.
"""
import json
import math
import os
import warnings

import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle import thermo

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
T_TEST = 0.06


def test_paper_cs_constants():
    g = GOLD["cs_eos"]
    assert (thermo.A_CS, thermo.B_CS, thermo.R_CS) == (g["a"], g["b"], g["R"])


def test_c_and_numpy_eos_agree():
    for rho in np.geomspace(1e-12, 0.9, 40):
        assert oracle.cs_p0(rho, T_TEST) == pytest.approx(float(thermo.p0(rho, T_TEST)), rel=1e-14, abs=1e-300)
        assert oracle.cs_mu0(rho, T_TEST) == pytest.approx(float(thermo.mu0(rho, T_TEST)), rel=1e-14)


def test_cs_virial_series():
    """Carnahan-Starling compressibility Z = p/(rho R T) of the repulsive part is
    1 + sum_{n>=1} (n^2 + 3n) eta^n (the textbook construction of the CS EOS).
    With a = 0, Eq. 20 must reproduce it."""
    for eta in (0.01, 0.05, 0.1):
        rho = 4 * eta / 4.0
        Z = oracle.cs_p0(rho, 1.0, 0.0, 4.0, 1.0) / rho
        series = 1.0 + sum((n * n + 3 * n) * eta ** n for n in range(1, 60))
        assert Z == pytest.approx(series, rel=1e-13)


def test_gibbs_duhem():
    """rho dmu0/drho = dp0/drho (Eqs. 7 and 9 with psi' = mu0): ties Eq. 21 to Eq. 20.
    Derivatives by 4-point central differences in log rho."""
    for rho in np.geomspace(1e-10, 0.85, 25):
        h = 2e-4
        def d(f):
            fp = lambda s: f(rho * math.exp(s))
            return (-fp(2 * h) + 8 * fp(h) - 8 * fp(-h) + fp(-2 * h)) / (12 * h) / rho
        dmu = d(lambda r: oracle.cs_mu0(r, T_TEST))
        dp = d(lambda r: oracle.cs_p0(r, T_TEST))
        assert rho * dmu == pytest.approx(dp, rel=1e-8, abs=1e-14)


def test_mu0_constant_as_printed():
    """Eq. 21's additive constant: mu0 - R T ln rho -> 4 R T as rho -> 0
    ((3 - 0)/1 + 1); Gibbs-Duhem cannot see it, but the upper limit of Sec. 5.6 can."""
    rho = 1e-14
    assert oracle.cs_mu0(rho, T_TEST) - T_TEST * math.log(rho) == pytest.approx(4 * T_TEST, rel=1e-12)


def test_dp0_drho_matches_fd():
    for rho in np.linspace(0.01, 0.8, 30):
        h = 1e-6
        fd = (oracle.cs_p0(rho + h, T_TEST) - oracle.cs_p0(rho - h, T_TEST)) / (2 * h)
        assert float(thermo.dp0_drho(rho, T_TEST)) == pytest.approx(fd, rel=1e-7, abs=1e-12)


def test_critical_point_definition():
    Tc, rc = thermo.critical_point()
    h = 1e-5
    p = lambda r: oracle.cs_p0(r, Tc)
    d1 = (p(rc + h) - p(rc - h)) / (2 * h)
    d2 = (p(rc + h) - 2 * p(rc) + p(rc - h)) / h ** 2
    assert abs(d1) < 1e-9 and abs(d2) < 1e-6
    # just above T_c p is monotone, just below it is not
    rs = np.linspace(0.05, 0.25, 2001)
    assert np.all(np.diff(thermo.p0(rs, 1.001 * Tc)) > 0)
    assert np.any(np.diff(thermo.p0(rs, 0.999 * Tc)) < 0)
    # CS critical packing fraction eta_c = b rho_c / 4 is universal (a, b, R free)
    Tc2, rc2 = thermo.critical_point(a=2.0, b=3.0, R=1.5)
    assert 3.0 * rc2 / 4 == pytest.approx(4.0 * rc / 4, rel=1e-10)


@pytest.mark.parametrize("T_r", [0.95, 0.7, 0.5, 0.35, 0.25])
def test_maxwell_equal_area(T_r):
    """Sec. 5.1 benchmark: equal pressure, equal chemical potential, and the
    equal-area rule  int_{v_l}^{v_g} p dv = p_sat (v_g - v_l),  v = 1/rho."""
    Tc, _ = thermo.critical_point()
    T = T_r * Tc
    rg, rl = thermo.maxwell(T_r)
    assert rg < rl
    # the gas-side pressure is the well-conditioned one (the liquid side is a
    # difference of two O(0.1) terms at low T)
    psat = oracle.cs_p0(rg, T)
    assert oracle.cs_p0(rl, T) == pytest.approx(psat, rel=1e-6, abs=2e-16)
    assert oracle.cs_mu0(rg, T) == pytest.approx(oracle.cs_mu0(rl, T), rel=1e-12, abs=1e-14)
    # equal area, integrated in s = ln v and split at the spinodals
    sg, sl = thermo.spinodals(T)
    f = lambda s: oracle.cs_p0(math.exp(-s), T) * math.exp(s)
    edges = [-math.log(rl), -math.log(sl), -math.log(sg), -math.log(rg)]
    area = sum(integrate.quad(f, a, b, limit=500, epsabs=0, epsrel=1e-13)[0]
               for a, b in zip(edges[:-1], edges[1:]))
    assert area == pytest.approx(psat * (1 / rg - 1 / rl), rel=1e-9)


def test_maxwell_mean_field_exponent():
    """Near T_c an analytic EOS gives rho_l - rho_g proportional to (1 - T_r)^(1/2)
    (the classical exponent beta = 1/2): the amplitude must settle."""
    Tc, rc = thermo.critical_point()
    amp = []
    for t in (0.999, 0.9999, 0.99999):
        g, l = thermo.maxwell(t)
        assert g < rc < l
        amp.append((l - g) / rc / math.sqrt(1 - t))
    assert amp[2] == pytest.approx(amp[1], rel=1e-4)
    assert amp[1] == pytest.approx(amp[0], rel=1e-3)


def test_density_ratio_claim_reachable():
    """Sec. 5.1 reports CS density ratios above 3.4e14; the Maxwell pair at
    T_r = 0.155 exceeds that."""
    rg, rl = thermo.maxwell(0.155)
    assert rl / rg > GOLD["cs_density_ratio_claim"]["value"]


def test_omega_double_roots():
    """The right side of Eq. 22 vanishes with zero slope at both bulk densities
    and is positive between them."""
    Tc, _ = thermo.critical_point()
    T = 0.6 * Tc
    rg, rl = thermo.maxwell(0.6)
    om = lambda r: float(thermo.omega(r, T, rl))
    assert abs(om(rg)) < 1e-14 and abs(om(rl)) < 1e-14
    assert all(om(r) > 0 for r in np.linspace(rg, rl, 50)[1:-1])
    h = 1e-6
    assert abs((om(rl + h) - om(rl - h)) / (2 * h)) < 1e-9


def test_sigma_matches_profile_integral():
    """sigma-hat from Eq. 24 integrated over rho equals kappa int (d rho/dy)^2 dy
    over the Eq. 23 profile; both scale as k (Sec. 5.2)."""
    s1 = thermo.sigma_flat(0.7, 0.1, 1.0)
    s2 = thermo.sigma_flat(0.7, 0.1, 0.5)
    assert s2 == pytest.approx(0.5 * s1, rel=1e-9)
    Tc, _ = thermo.critical_point()
    rg, rl = thermo.maxwell(0.7)
    rs = np.linspace(rg, rl, 4001)[1:-1]
    y = thermo.flat_profile_y(rs[::40], 0.7, 0.1, 1.0)
    # kappa (drho/dy)^2 dy = kappa drho/dy drho
    grad = thermo.flat_gradient(rs, 0.7 * Tc, rl, 0.1, 1.0)
    s3 = np.trapezoid(0.1 * grad, rs)
    assert s3 == pytest.approx(s1, rel=1e-4)
    assert np.all(np.diff(y) > 0)


def test_laplace_pair_limits():
    """Large drops recover the flat Maxwell pair; the gas density rises for small drops."""
    rg, rl = thermo.maxwell(0.6)
    g1, l1 = thermo.laplace_pair(0.6, 0.1, 0.5, 1e7)
    assert g1 == pytest.approx(rg, rel=1e-5) and l1 == pytest.approx(rl, rel=1e-6)
    g2, l2 = thermo.laplace_pair(0.6, 0.1, 0.5, 20)
    assert g2 > rg and l2 > rl


def test_laplace_pair_against_gibbs_duhem_quadrature():
    """The drop pair at one radius, found another way.  Along each stable branch
    the pressure follows Gibbs-Duhem, dp = rho dmu, so from the Maxwell point the
    jump grows as integral_{mu_M}^{mu} (rho_l(m) - rho_g(m)) dm, with each
    branch's rho(m) found by inverting Eq. 21 alone (Newton on the branch, no
    Eq. 20).  The pair is where that jump, moved to the mesh space by k^2
    (Eq. 29), equals sigma-hat / R (Eq. 40), with sigma-hat the profile integral
    kappa-hat int (d rho/dy)^2 dy over the Eq. 23 profile (Eq. 10).  A wrong k^2
    on the jump, a wrong sigma or a pressure that is not Eq. 20's would move it."""
    Tr, kappa, k, radius = 0.6, 0.1, 0.5, 40.0
    Tc, _ = thermo.critical_point()
    T = Tr * Tc
    rg, rl = thermo.maxwell(Tr)
    # sigma-hat as the profile integral kappa int (d rho/dy) d rho, with the slope
    # taken by differences of the Eq. 23 coordinate y(rho), trapezoid rule
    mid = 0.5 * (rg + rl)
    rho_grid = np.concatenate([rg + np.geomspace(1e-6 * rg, mid - rg, 300),
                               (rl - np.geomspace(rl - mid, 1e-7 * rl, 300))[1:]])
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        y = thermo.flat_profile_y(rho_grid, Tr, kappa, k)
    slope = 1.0 / np.gradient(y, rho_grid)
    sigma = kappa * float(np.sum(0.5 * (slope[1:] + slope[:-1]) * np.diff(rho_grid)))
    assert sigma == pytest.approx(thermo.sigma_flat(Tr, kappa, k), rel=3e-3)
    target = sigma / radius / (k * k)

    def mu(r):
        return float(thermo.mu0(r, T))

    def branch(m, r_start):  # Newton on Eq. 21 in log rho (numerical derivative)
        s = math.log(r_start)
        for _ in range(60):
            h = 1e-6
            f = mu(math.exp(s)) - m
            fp = (mu(math.exp(s + h)) - mu(math.exp(s - h))) / (2 * h)
            step = f / fp
            s -= step
            if abs(step) < 1e-15:
                break
        return math.exp(s)

    mu_M = mu(rg)
    nodes, weights = np.polynomial.legendre.leggauss(24)

    def jump(m):  # integral of (rho_l - rho_g) dm from mu_M to m, Gauss-Legendre
        ms = mu_M + 0.5 * (m - mu_M) * (nodes + 1)
        vals = [branch(x, rl) - branch(x, rg) for x in ms]
        return 0.5 * (m - mu_M) * float(np.dot(weights, vals))

    lo, hi = mu_M, mu_M + 2 * target / (rl - rg)
    for _ in range(60):  # bisection on the chemical potential
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if jump(mid) < target else (lo, mid)
    m = 0.5 * (lo + hi)
    g_ref, l_ref = branch(m, rg), branch(m, rl)
    g, l = thermo.laplace_pair(Tr, kappa, k, radius)
    # both routes agree on the shift from Maxwell to the quadrature's accuracy
    # (9e-4 of the shift measured, from sigma's trapezoid rule)
    assert abs(g - g_ref) <= 3e-3 * (g_ref - rg)
    assert abs(l - l_ref) <= 3e-3 * (l_ref - rl)
    # and the shift itself is well resolved: a few percent on the gas
    assert 0.005 < g / rg - 1 < 0.2
