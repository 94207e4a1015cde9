"""Pins of the oracle's other equations of state (oracle/eos.py, the C oracle's
orc_p0/orc_mu0): VDW (Eqs. 14-15), RK and RKS (Eqs. 16-17), PR (Eqs. 18-19),
with CS (Eqs. 20-21) by the same generic route.

  * Gibbs-Duhem: each printed mu0 must satisfy rho d(mu0)/d(rho) = d(p0)/d(rho)
    with its printed p0 (Eqs. 7, 9, 13), by independent central differences;
  * critical points against closed forms: VDW T_c = 8a/(27Rb), rho_c = 1/(3b);
    RK/RKS Omega_b = b p_c/(R T_c) = (2^(1/3) - 1)/3, Omega_a = 1/(9(2^(1/3) - 1)),
    Z_c = 1/3; PR Omega_b = 0.0777960739, Omega_a = 0.4572355289, Z_c = 0.3074013;
  * alpha(T_c) = 1 for RKS and PR (their alpha is written in T_r);
  * the Maxwell pair obeys the equal-area rule by quadrature, and the generic
    solver reproduces the dedicated CS solver of oracle/thermo.py;
  * the C oracle's p0 and mu0 equal the Python ones.
"""

import numpy as np
import pytest
from scipy import integrate

from oracle import eos as E
from oracle import sim as S
from oracle import thermo

OMEGA = {"rks": 0.344, "pr": 0.344}


def mk(kind, **kw):
    return E.Eos(kind, omega=OMEGA.get(kind, 0.0), **kw)


@pytest.mark.parametrize("kind", E.KINDS)
@pytest.mark.parametrize("t_r", [0.5, 0.8, 1.2])
def test_gibbs_duhem(kind, t_r):
    e = mk(kind)
    tc, rc = e.critical_point()
    T = t_r * tc
    for r in np.linspace(0.05 * rc, 0.92 * e.rho_max, 9):
        h = 1e-5 * r
        dmu = (e.mu0(r + h, T) - e.mu0(r - h, T)) / (2 * h)
        dp = (e.p0(r + h, T) - e.p0(r - h, T)) / (2 * h)
        assert r * dmu == pytest.approx(dp, rel=1e-6, abs=1e-9 * abs(e.p0(r, T)) + 1e-14)


@pytest.mark.parametrize("a,b", [(9 / 49, 2 / 21), (0.5, 0.3)])
def test_vdw_critical_closed_form(a, b):
    tc, rc = E.Eos("vdw", a=a, b=b).critical_point()
    assert tc == pytest.approx(8 * a / (27 * b), rel=1e-12)
    assert rc == pytest.approx(1 / (3 * b), rel=1e-7)


@pytest.mark.parametrize("kind", ["rk", "rks"])
def test_redlich_kwong_critical_constants(kind):
    e = mk(kind)
    tc, rc = e.critical_point()
    al = e.alpha(tc)
    pc = e.p0(rc, tc, al)
    c = 2 ** (1 / 3) - 1
    assert e.b * pc / (e.R * tc) == pytest.approx(c / 3, rel=1e-12)
    assert e.a * al * pc / (e.R * tc) ** 2 == pytest.approx(1 / (9 * c), rel=1e-12)
    assert pc / (rc * e.R * tc) == pytest.approx(1 / 3, rel=1e-7)


def test_peng_robinson_critical_constants():
    e = mk("pr")
    tc, rc = e.critical_point()
    pc = e.p0(rc, tc)
    assert e.alpha(tc) == 1.0
    assert e.b * pc / (e.R * tc) == pytest.approx(0.0777960739, rel=1e-9)
    assert e.a * pc / (e.R * tc) ** 2 == pytest.approx(0.4572355289, rel=1e-9)
    assert pc / (rc * e.R * tc) == pytest.approx(0.3074013, rel=1e-6)


@pytest.mark.parametrize("kind", ["rks", "pr"])
def test_alpha_is_one_at_tc_and_falls_with_t(kind):
    e = mk(kind)
    tc, _ = e.critical_point()
    assert e.alpha(tc) == 1.0
    assert e.alpha(0.5 * tc) > e.alpha(0.8 * tc) > 1.0 > e.alpha(1.2 * tc)
    assert E.Eos("rk").alpha(0.25) == 2.0


@pytest.mark.parametrize("kind", E.KINDS)
@pytest.mark.parametrize("t_r", [0.8, 0.6])
def test_equal_area(kind, t_r):
    """Maxwell: the integral of p0 dv over the loop equals p_sat (v_g - v_l),
    v = 1/rho, i.e. int p0/rho^2 d rho from rho_g to rho_l."""
    e = mk(kind)
    tc, _ = e.critical_point()
    T = t_r * tc
    rg, rl = e.maxwell(t_r)
    ps = e.p0(rg, T)
    assert e.p0(rl, T) == pytest.approx(ps, rel=1e-9)
    assert e.mu0(rl, T) == pytest.approx(e.mu0(rg, T), rel=1e-9, abs=1e-12)
    sg, sl = e.spinodals(T)
    f = lambda r: e.p0(r, T) / r**2
    area = sum(integrate.quad(f, lo, hi, epsabs=0, epsrel=1e-13, limit=400)[0]
               for lo, hi in ((rg, sg), (sg, sl), (sl, rl)))
    assert area == pytest.approx(ps * (1 / rg - 1 / rl), rel=1e-8)


@pytest.mark.parametrize("t_r", [0.9, 0.6, 0.4])
def test_generic_cs_matches_dedicated_solver(t_r):
    g, l = mk("cs").maxwell(t_r)
    tg, tl = thermo.maxwell(t_r)
    assert g == pytest.approx(tg, rel=1e-10) and l == pytest.approx(tl, rel=1e-12)
    assert mk("cs").critical_point()[0] == pytest.approx(thermo.critical_point()[0], rel=1e-12)


@pytest.mark.parametrize("kind", E.KINDS)
def test_c_oracle_matches_python(kind):
    e = mk(kind)
    tc, rc = e.critical_point()
    T = 0.6 * tc
    al = e.alpha(T)
    for r in (0.2 * rc, rc, 0.85 * e.rho_max):
        assert S.eos_p0(kind, r, T, e.a, e.b, e.R, al) == pytest.approx(e.p0(r, T), rel=1e-13,
                                                                         abs=1e-16)
        assert S.eos_mu0(kind, r, T, e.a, e.b, e.R, al) == pytest.approx(e.mu0(r, T),
                                                                          rel=1e-13, abs=1e-16)


@pytest.mark.parametrize("kind", E.KINDS)
def test_mu0_grows_without_bound_below_the_pole(kind):
    """The repulsive pole (b rho = 1, or b rho / 4 = 1 for CS): approached from
    below, mu0 rises past any bound, so +infinity is its value there."""
    e = mk(kind)
    T = 0.6 * e.critical_point()[0]
    pole = 1.0 / (e.b / 4.0 if kind == "cs" else e.b)
    vals = [e.mu0(pole * (1 - d), T) for d in (1e-2, 1e-4, 1e-6, 1e-8)]
    assert all(np.diff(vals) > 0) and vals[-1] > 10 * abs(vals[0])


@pytest.mark.parametrize("kind", ["cs", "pr"])
def test_upper_limit_replaces_mu_at_the_pole(kind):
    """Sec. 5.6: while the limit is active, a node at or beyond the pole (where
    the chemical potential overflows) gets mu-hat = k^2 mu_max and its
    neighbours stay finite; without the limit mu-hat is infinite there."""
    from oracle import OracleSim
    e = None if kind == "cs" else mk(kind)
    ee = mk(kind)
    tc = ee.critical_point()[0]
    rg, rl = ee.maxwell(0.6)
    pole = 1.0 / (ee.b / 4.0 if kind == "cs" else ee.b)
    kappa, k, mu_max = (0.1, 0.5, 2.0) if kind == "cs" else (0.005, 0.2, 6.0)
    rho = np.full((12, 16), rl)
    rho[5, 7] = 1.02 * pole
    rho[6, 7] = pole
    capped = OracleSim(16, 12, 0.6 * tc, kappa, 1.0, k, 6, eos=e, mu_max=mu_max,
                       mu_cap_steps=10)
    mu, Fx, Fy = capped.force_stage(rho, t=0)
    assert mu[5, 7] == k * k * mu_max and mu[6, 7] == k * k * mu_max
    assert np.isfinite(mu).all() and np.isfinite(Fx).all() and np.isfinite(Fy).all()
    free = OracleSim(16, 12, 0.6 * tc, kappa, 1.0, k, 6, eos=e)
    mu, _, _ = free.force_stage(rho, t=0)
    assert mu[5, 7] == np.inf and mu[6, 7] == np.inf


def test_pr_and_rks_density_ratio_at_tr_0_4_exceeds_the_printed_bound():
    """Sec. 5.4 (Fig. 9b): at T_r 0.4 the PR and RKS density ratios exceed
    65,000 (tests/golden/paper_constants.json).  The Maxwell pairs give
    6.8e5 and 7.5e5."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "paper_constants.json")))["pr_rks_ratio_at_tr_0_4"]
    for kind in ("pr", "rks"):
        g, l = E.Eos(kind, omega=gold["omega"]).maxwell(gold["T_r"])
        assert l / g > gold["value"], (kind, l / g)


@pytest.mark.parametrize("kind,t_r", [("vdw", 0.12), ("pr", 0.2), ("rks", 0.2)])
def test_printed_maximum_density_ratios_are_reachable(kind, t_r):
    """Sec. 5.1 reports density ratios above 5.5e10 (VDW), 6.9e11 (PR) and
    2.8e13 (RKS); the oracle's Maxwell pair passes each at the given T_r
    (5.8e10, 9.5e15 and 2.7e16), with finite, ordered densities."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "paper_constants.json")))["max_density_ratio_claims"]
    e = E.Eos(kind, omega=gold["omega"] if kind != "vdw" else 0.0)
    g, l = e.maxwell(t_r)
    assert 0 < g < l < e.rho_max and l / g > gold[kind]
