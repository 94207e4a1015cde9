"""The oracle against the paper's physical invariants (Secs. 5.1, 5.3-5.5), on
CPU at sizes the plain C oracle finishes in seconds.  The Maxwell pair and the
flat-interface tension these compare with come from oracle/thermo.py, pinned
by closed forms in test_oracle_lbm.py and test_oracle_eos_variants.py.

  * flat coexistence (Sec. 5.1): the liquid settles on the Maxwell density; the
    gas settles slightly above it, by the discrete scheme's offset (+0.65% at
    T_r 0.8, k 0.3), which the paper's logarithmic axis does not resolve;
  * the discrete equilibrium law: at rest (v = 0, so u = -F/(2 rho)) the
    exact-difference forcing of Eq. 5 with D2Q9 streaming balances momentum as
      F = c_s^2 d_c rho + d_c(F^2/(4 rho)) - d2 F / 4
    (d_c the central difference, d2 the second difference); with F from Eq.
    12 and the compact derivative D, and expanding in the interface width,
      mu-hat - (c_s^4/4) [rho''/rho - rho'^2/(2 rho^2)] = const,
    so the flat profile is that of Eq. 23 with kappa-hat replaced by
    kappa_eff(rho) = kappa-hat + c_s^4/(4 rho).  The oracle's flat profile
    approaches it at second order in k (error 2.8e-3 of rho_l - rho_g at
    k 0.4, 6.7e-4 at 0.2, 1.6e-4 at 0.1), for any tau and under MRT, while
    Eq. 23 with the nominal kappa-hat stays 14% away at every k.  A slab at 45
    degrees to the grid follows the same law along its normal (1.5e-3 at
    k 0.5): the law is isotropic at this order.  It does not depend on the EOS:
    a PR slab (T_r 0.7, kappa-hat 0.005, k 0.3), where c_s^4/(4 rho) is ten to
    twenty times kappa-hat on the gas side, follows it to 2.7e-3 (15% with the
    nominal kappa-hat).  Started from Eq. 23's profile
    with the nominal kappa-hat (T_r 0.5, k 0.2), the gas goes negative in the
    first step; from the law's profile the run starts cleanly;
  * Young-Laplace (Sec. 5.3): Delta P R is the same for drops of radius 12 and
    15, and equals the tension of that law, the integral of
    sqrt(2 k^2 Omega(rho) kappa_eff(rho)) d rho (Eq. 24 with kappa_eff), to 3%
    (measured 1.2% and 2.2%; Eq. 24 with the nominal kappa-hat is 1.76 times
    smaller).  The paper's integral method (Fig. 8), P_N - P_T integrated
    along the vertical line through the drop centre, agrees with it to 3% when
    P_N - P_T is the scheme's kappa_eff(rho) rho'^2 (measured 1.0% and 1.8%);
    with kappa-hat rho'^2 it is 2.9 times smaller;
  * spurious current (Sec. 5.4): below 1e-3 at equilibrium (measured 3.1e-4 at
    T_r 0.7, k 0.25), and larger at lower temperature (Fig. 9a): 6.8e-5, 2.7e-4
    and 9.7e-4 at T_r 0.8, 0.7 and 0.6 for a drop of radius 16 on 64^2;
  * Galilean invariance (Sec. 5.5): a drop advected at 0.05 for 400 steps moves
    by 20 nodes and keeps the static drop's outline;
  * independence of the relaxation time (Sec. 5.1): the MRT model at tau 0.8 and
    the single-relaxation-time model at tau 3.0 settle on the same coexistence
    densities (here to 1e-6);
  * the interface width is inversely proportional to k and the mesh-space
    tension proportional to it (Sec. 5.2, Figs. 6-7): at k 0.1 the 10-90% width
    is twice and kappa-hat * sum (d rho/dy)^2 half that at k 0.2, to 5%;
  * the chemical potential is constant in the bulk phases at equilibrium (Sec.
    5.1): within each bulk of a flat interface to 1e-6 (measured 2e-7 in the gas,
    3e-10 in the liquid; |mu-hat| is 5e-3).
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import OracleSim, thermo
from paper_1906_09530_gb300 import workloads as W

pytestmark = pytest.mark.slow
TC, _ = thermo.critical_point()


def test_flat_coexistence_against_maxwell():
    tr, k, ny = 0.8, 0.3, 100
    rg, rl = thermo.maxwell(tr)
    o = OracleSim(8, ny, tr * TC, 0.1, 1.0, k, 6)
    o.set_fields(W.flat(8, ny, rg, rl, ny / 2, 4.0 / k))
    o.step(10_000)
    r = o.fields()[0][:, 0]
    gas = np.r_[r[:10], r[-10:]].mean()
    liq = r[ny // 2 - 10: ny // 2 + 10].mean()
    assert abs(liq / rl - 1) <= 1e-4
    assert 0 < gas / rg - 1 <= 1e-2


def _drop_state(n, T, k, R, steps, width=4.0):
    rg, rl = thermo.maxwell(T / TC)
    o = OracleSim(n, n, T, 0.1, 1.0, k, 6)
    o.set_fields(W.drop(n, n, rg, rl, R, width))
    o.step(steps)
    return o.fields()[:3], rg, rl


CS4_4 = (1.0 / 3.0) ** 2 / 4.0  # c_s^4 / 4 = 1/36


def _kappa_eff(rho, kappa):
    return kappa + CS4_4 / rho


def _profile_y(rho_values, tr, kappa, k, kappa_of_rho):
    """y(rho) of a flat interface whose gradient coefficient is kappa_of_rho:
    (kappa(rho)/2)(d rho/dy)^2 = k^2 Omega(rho), integrated from the midpoint
    density (Eq. 23's quadrature with a density-dependent kappa)."""
    T = tr * TC
    rg, rl = thermo.maxwell(tr)
    r0 = 0.5 * (rg + rl)
    out = []
    for r in rho_values:
        f = lambda s: 1.0 / thermo.flat_gradient(s, T, rl, kappa_of_rho(s, kappa), k)  # noqa: E731
        v, _ = integrate.quad(f, r0, r, limit=400, epsabs=0, epsrel=1e-11)
        out.append(v)
    return np.array(out)


def _sigma_law(tr, kappa, k, kappa_of_rho):
    T = tr * TC
    rg, rl = thermo.maxwell(tr)
    f = lambda r: math.sqrt(max(2 * k * k * float(thermo.omega(r, T, rl)) *  # noqa: E731
                                kappa_of_rho(r, kappa), 0.0))
    v, _ = integrate.quad(f, rg, rl, points=np.geomspace(rg, rl, 12)[1:-1], limit=400,
                          epsabs=0, epsrel=1e-11)
    return v


def test_flat_profile_follows_the_discrete_equilibrium_law():
    tr, kappa = 0.8, 0.1
    rg, rl = thermo.maxwell(tr)
    rs = np.linspace(rg, rl, 1202)[1:-1]
    errs = {}
    for k, ny, steps in ((0.4, 80, 10_000), (0.2, 160, 30_000)):
        o = OracleSim(4, ny, tr * TC, kappa, 1.0, k, 6)
        o.set_fields(W.flat(4, ny, rg, rl, ny / 2, 4.0 / k))
        o.step(steps)
        half = o.fields()[0][: ny // 2, 0]
        mid = 0.5 * (rg + rl)
        i = int(np.argmax(half >= mid))
        y = np.arange(ny // 2) - ((i - 1) + (mid - half[i - 1]) / (half[i] - half[i - 1]))
        for name, kap in (("eff", _kappa_eff), ("nominal", lambda r, c: c)):
            ys = _profile_y(rs, tr, kappa, k, kap)
            sel = (y > ys[0]) & (y < ys[-1])
            errs[k, name] = np.abs(half[sel] - np.interp(y[sel], ys, rs)).max() / (rl - rg)
    assert errs[0.4, "eff"] <= 4e-3 and errs[0.2, "eff"] <= 1e-3, errs
    assert errs[0.4, "eff"] / errs[0.2, "eff"] >= 3.0, errs  # second order in k
    assert errs[0.4, "nominal"] >= 0.1 and errs[0.2, "nominal"] >= 0.1, errs


def test_peng_robinson_slab_follows_the_same_law():
    from oracle import eos as E
    e = E.Eos("pr", omega=0.344)
    tr, kappa, k, ny = 0.7, 0.005, 0.3, 160
    T = tr * e.critical_point()[0]
    rg, rl = e.maxwell(tr)
    mu_b = e.mu0(rl, T)

    def omega(r):  # right side of Eq. 22 with the PR psi
        return r * (e.mu0(r, T) - mu_b) - (e.p0(r, T) - e.p0(rl, T))

    def profile_y(rs, kap):
        r0, out = 0.5 * (rg + rl), []
        for r in rs:
            f = lambda s_: 1.0 / math.sqrt(max(2 * k * k * omega(s_) / kap(s_), 1e-300))  # noqa
            out.append(integrate.quad(f, r0, r, limit=400, epsabs=0, epsrel=1e-10)[0])
        return np.array(out)

    o = OracleSim(4, ny, T, kappa, 1.0, k, 6, eos=e)
    o.set_fields(W.flat(4, ny, rg, rl, ny / 2, 4.0 / k))
    o.step(20_000)
    half = o.fields()[0][: ny // 2, 0]
    mid = 0.5 * (rg + rl)
    i = int(np.argmax(half >= mid))
    y = np.arange(ny // 2) - ((i - 1) + (mid - half[i - 1]) / (half[i] - half[i - 1]))
    rs = np.linspace(rg, rl, 1202)[1:-1]
    errs = []
    for kap in (lambda r: _kappa_eff(r, kappa), lambda r: kappa):
        ys = profile_y(rs, kap)
        sel = (y > ys[0]) & (y < ys[-1])
        errs.append(np.abs(half[sel] - np.interp(y[sel], ys, rs)).max() / (rl - rg))
    assert errs[0] <= 5e-3 and errs[1] >= 0.1, errs


def test_diagonal_slab_follows_the_same_law():
    tr, kappa, k, n = 0.8, 0.1, 0.5, 64
    rg, rl = thermo.maxwell(tr)
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    s = (x + y) % n  # the normal distance is s / sqrt(2)
    rho = rg + (rl - rg) * 0.5 * (1 - np.tanh(2 * (np.abs(s - n / 2) - n / 4) / np.sqrt(2)
                                              / (4.0 / k)))
    o = OracleSim(n, n, tr * TC, kappa, 1.0, k, 6)
    o.set_fields(rho)
    o.step(4000)
    r = o.fields()[0]
    assert np.abs(r - np.roll(np.roll(r, 1, axis=0), -1, axis=1)).max() <= 1e-12  # still 1-D
    half = r[0, : n // 2]
    mid = 0.5 * (rg + rl)
    i = int(np.argmax(half >= mid))
    d = (np.arange(n // 2) - ((i - 1) + (mid - half[i - 1]) / (half[i] - half[i - 1]))) \
        / np.sqrt(2)
    rs = np.linspace(rg, rl, 1202)[1:-1]
    errs = []
    for kap in (_kappa_eff, lambda r_, c: c):
        ys = _profile_y(rs, tr, kappa, k, kap)
        sel = (d > ys[0]) & (d < ys[-1])
        errs.append(np.abs(half[sel] - np.interp(d[sel], ys, rs)).max() / (rl - rg))
    assert errs[0] <= 3e-3 and errs[1] >= 0.1, errs


def test_nominal_eq23_start_fails_and_the_law_start_does_not():
    tr, kappa, k, ny = 0.5, 0.1, 0.2, 384
    rg, rl = thermo.maxwell(tr)
    rs = np.linspace(rg, rl, 4002)[1:-1]
    d = ny / 4.0 - np.abs(np.arange(ny, dtype=np.float64) - ny / 2.0)  # > 0 in the liquid
    mins = []
    for kap in (lambda r_, c: c, _kappa_eff):
        col = np.interp(d, _profile_y(rs, tr, kappa, k, kap), rs, left=rg, right=rl)
        o = OracleSim(4, ny, tr * TC, kappa, 1.0, k, 6)
        o.set_fields(np.repeat(col[:, None], 4, axis=1))
        o.step(1)
        mins.append(o.fields()[0].min())
        if kap is _kappa_eff:
            o.step(199)
            r = o.fields()[0]
            assert np.isfinite(r).all() and r.min() > 0.5 * rg
    assert mins[0] < 0 < mins[1], mins


def test_laplace_law():
    tr, k, n = 0.7, 0.5, 48
    T = tr * TC
    y, x = np.mgrid[0:n, 0:n]
    d = np.hypot(x - n / 2, y - n / 2)
    prod, R_eff, dP_all, integral, integral_nominal = [], [], [], [], []
    deriv = OracleSim(n, n, T, 0.1, 1.0, k, 6)  # for the compact y-derivative only
    for R in (12.0, 15.0):
        (rho, _, _), rg, rl = _drop_state(n, T, k, R, 3000)
        Ri = math.sqrt((rho > 0.5 * (rg + rl)).sum() / math.pi)
        rin = rho[d < 0.5 * Ri].mean()
        rout = rho[d > Ri + 0.5 * (n / 2 - Ri)].mean()
        dP = k * k * (thermo.p0(rin, T) - thermo.p0(rout, T))
        prod.append(dP * Ri)
        R_eff.append(Ri)
        dP_all.append(dP)
        col = rho[: n // 2, n // 2]  # the lower crossing of the vertical centre line
        dcol = deriv.cfd_field(rho, 1)[: n // 2, n // 2]
        integral.append(np.sum(_kappa_eff(col, 0.1) * dcol ** 2))
        integral_nominal.append(np.sum(0.1 * dcol ** 2))
    assert dP_all[0] > dP_all[1] > 0
    assert abs(prod[0] / prod[1] - 1) <= 0.02
    sigma_eff = _sigma_law(tr, 0.1, k, _kappa_eff)
    assert all(abs(p / sigma_eff - 1) <= 0.03 for p in prod), (prod, sigma_eff)
    assert all(abs(p / s - 1) <= 0.03 for p, s in zip(prod, integral)), (prod, integral)
    assert all(2.5 <= p / s <= 3.3 for p, s in zip(prod, integral_nominal))
    assert sigma_eff / _sigma_law(tr, 0.1, k, lambda r, c: c) == pytest.approx(1.76, rel=0.02)


def test_spurious_current():
    tr, k, n = 0.7, 0.25, 96
    (rho, vx, vy), _, _ = _drop_state(n, tr * TC, k, 24.0, 4000, width=4.0 / k)
    assert np.hypot(vx, vy).max() < 1e-3


def test_spurious_current_grows_as_temperature_falls():
    n, k = 64, 0.25
    vmax = []
    for tr in (0.8, 0.7, 0.6):
        rg, rl = thermo.maxwell(tr)
        o = OracleSim(n, n, tr * TC, 0.1, 1.0, k, 6)
        o.set_fields(W.drop(n, n, rg, rl, 16.0, 4.0 / k))
        o.step(2000)
        vmax.append(np.hypot(*o.fields()[1:3]).max())
    # measured 6.8e-5, 2.7e-4, 9.7e-4: the claim is the growth, each at least
    # twice the one above it; the bound only keeps the level in the regime of
    # Sec. 5.4, with room for step-count and rounding changes
    assert vmax[0] * 2 < vmax[1] and vmax[1] * 2 < vmax[2] < 2e-3, vmax


def test_galilean_translation():
    tr, k, n, u0, steps = 0.7, 0.5, 32, 0.05, 400
    T = tr * TC
    rg, rl = thermo.maxwell(tr)
    out = []
    for u in (0.0, u0):
        o = OracleSim(n, n, T, 0.1, 1.0, k, 6)
        rho = W.drop(n, n, rg, rl, 8.0, 4.0)
        o.set_fields(rho, np.full_like(rho, u), np.zeros_like(rho))
        o.step(steps)
        out.append(o.fields()[0])

    def centre_x(r):  # centre of the excess mass along the periodic x axis
        w = (r - rg).sum(axis=0)
        ang = 2 * np.pi * np.arange(n) / n
        return (np.angle((w * np.exp(1j * ang)).sum()) / (2 * np.pi) * n) % n

    static, moved = out
    shift = (centre_x(moved) - centre_x(static)) % n
    assert abs(shift - u0 * steps) <= 0.5
    back = np.roll(moved, -int(round(u0 * steps)), axis=1)
    mid = 0.5 * (rg + rl)
    ps, pm = static > mid, back > mid
    links = (np.diff(ps.astype(np.int8), axis=1) != 0).sum() + \
        (np.diff(ps.astype(np.int8), axis=0) != 0).sum()
    assert (ps != pm).sum() <= 0.25 * links


def _flat_bulks(tr, k, ny, tau, steps, mrt=None):
    from oracle import sim as S
    rg, rl = thermo.maxwell(tr)
    o = OracleSim(8, ny, tr * TC, 0.1, tau, k, 6, mrt=S.PAPER_MRT if mrt else None)
    o.set_fields(W.flat(8, ny, rg, rl, ny / 2, 4.0 / k))
    o.step(steps)
    return o.fields()[0][:, 0]


def test_coexistence_independent_of_relaxation_time():
    ny = 64
    a = _flat_bulks(0.7, 0.3, ny, 3.0, 20_000)
    b = _flat_bulks(0.7, 0.3, ny, 0.8, 20_000, mrt=True)
    for r in (a, b):
        assert np.isfinite(r).all()
    ga, la = np.r_[a[:6], a[-6:]].mean(), a[ny // 2 - 6: ny // 2 + 6].mean()
    gb, lb = np.r_[b[:6], b[-6:]].mean(), b[ny // 2 - 6: ny // 2 + 6].mean()
    assert abs(ga / gb - 1) <= 1e-6 and abs(la / lb - 1) <= 1e-6


def _width_10_90(r):
    n = r.size
    g = np.r_[r[:10], r[-10:]].mean()
    l = r[n // 2 - 10: n // 2 + 10].mean()
    half = r[: n // 2]

    def cross(v):
        i = int(np.argmax(half >= v))
        return (i - 1) + (v - half[i - 1]) / (half[i] - half[i - 1])
    return cross(g + 0.9 * (l - g)) - cross(g + 0.1 * (l - g))


def _sigma(r, kappa=0.1):
    """kappa-hat times the sum of (d rho / dy)^2 over one interface (Eq. 24's
    integral over the measured profile, central differences)."""
    d = np.gradient(r[: r.size // 2 + 1])
    return kappa * np.sum(d * d)


def test_interface_width_and_tension_scale_with_k():
    """Width proportional to 1/k and the mesh-space tension to k, so both are
    the same in the momentum space (Sec. 5.2, Figs. 6-7)."""
    r2 = _flat_bulks(0.6, 0.2, 200, 1.0, 10_000)
    r1 = _flat_bulks(0.6, 0.1, 400, 1.0, 10_000)
    w2, w1 = _width_10_90(r2), _width_10_90(r1)
    assert abs(w1 / w2 / 2 - 1) <= 0.05, (w1, w2)
    assert abs(_sigma(r2) / _sigma(r1) / 2 - 1) <= 0.05


def test_chemical_potential_constant_in_each_bulk():
    tr, k, ny = 0.7, 0.3, 160
    rg, rl = thermo.maxwell(tr)
    o = OracleSim(8, ny, tr * TC, 0.1, 1.0, k, 6)
    o.set_fields(W.flat(8, ny, rg, rl, ny / 2, 4.0 / k))
    o.step(20_000)
    mu = o.fields()[3][:, 0]
    gas = np.r_[mu[:10], mu[-10:]]
    liq = mu[ny // 2 - 10: ny // 2 + 10]
    assert np.ptp(gas) <= 1e-6 and np.ptp(liq) <= 1e-6

