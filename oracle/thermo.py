"""Thermodynamics of the Carnahan-Starling fluid, plain FP64 numpy/scipy.

TEST INFRASTRUCTURE ONLY (part of the oracle): only the tests, the smoke check
and the benchmark's CPU-baseline leg use it.  Shares no code with the CUDA
library.

What it computes, each from its definition in the paper:
  * p0, mu0                   Eqs. 20-21 (a=1, b=4, R=1 by default, Sec. 3.2)
  * psi = rho*mu0 - p0        Eq. 9 solved for psi (the bulk free-energy density)
  * the critical point        top of the spinodal dp0/drho = 0 (Sec. 3.2, T_r = T/T_c)
  * Maxwell coexistence       equal pressure and equal chemical potential (Sec. 5.1)
  * the flat interface        Eqs. 22-24, in the mesh space of Eq. 33
  * flat surface tension      sigma-hat = integral of kappa-hat (d rho/dy)^2 dy
  * Laplace-shifted pair      bulk densities of a drop of radius R (Eq. 40)
"""
import math

import numpy as np
from scipy import integrate, optimize

A_CS, B_CS, R_CS = 1.0, 4.0, 1.0


def p0(rho, T, a=A_CS, b=B_CS, R=R_CS):
    """Carnahan-Starling pressure, Eq. 20."""
    eta = b * np.asarray(rho, dtype=np.float64) / 4.0
    return rho * R * T * (1 + eta + eta**2 - eta**3) / (1 - eta) ** 3 - a * rho**2


def mu0(rho, T, a=A_CS, b=B_CS, R=R_CS):
    """Carnahan-Starling chemical potential without the gradient term, Eq. 21."""
    eta = b * np.asarray(rho, dtype=np.float64) / 4.0
    return R * T * ((3 - eta) / (1 - eta) ** 3 + np.log(rho) + 1) - 2 * a * rho


def psi(rho, T, a=A_CS, b=B_CS, R=R_CS):
    """Bulk free-energy density from Eq. 9: psi = rho*psi' - p0 with psi' = mu0."""
    return rho * mu0(rho, T, a, b, R) - p0(rho, T, a, b, R)


def dp0_drho(rho, T, a=A_CS, b=B_CS, R=R_CS):
    """d p0 / d rho of Eq. 20.  With Z(eta) the bracket of Eq. 20 and
    eta = b rho/4, d(rho Z)/d rho = Z + eta Z'(eta)
      = (1 + 4 eta + 4 eta^2 - 4 eta^3 + eta^4) / (1 - eta)^4."""
    eta = b * np.asarray(rho, dtype=np.float64) / 4.0
    G = (1 + 4 * eta + 4 * eta**2 - 4 * eta**3 + eta**4) / (1 - eta) ** 4
    return R * T * G - 2 * a * rho


def critical_point(a=A_CS, b=B_CS, R=R_CS):
    """(T_c, rho_c): the top of the spinodal curve.  A density rho lies on the
    spinodal at the temperature T_sp(rho) that makes dp0/drho = 0, i.e.
    T_sp = 2 a rho / (R G(eta)) with G from dp0_drho; the critical point is the
    maximum of T_sp, located as the root of dT_sp/d eta, which is taken by the
    complex-step derivative (exact to rounding for this analytic function)."""
    def tsp(eta):
        rho = 4 * eta / b
        G = (1 + 4 * eta + 4 * eta**2 - 4 * eta**3 + eta**4) / (1 - eta) ** 4
        return 2 * a * rho / (R * G)
    h = 1e-30
    dT = lambda eta: (tsp(complex(eta, h)).imag) / h
    res = optimize.minimize_scalar(lambda e: -tsp(e), bounds=(1e-6, 0.9),
                                   method="bounded", options={"xatol": 1e-10})
    eta_c = optimize.brentq(dT, res.x - 1e-3, res.x + 1e-3, xtol=1e-16, rtol=1e-15)
    return float(tsp(eta_c)), 4 * eta_c / b


def spinodals(T, a=A_CS, b=B_CS, R=R_CS):
    """(rho_sp_gas, rho_sp_liq): the two roots of dp0/drho = 0 below T_c."""
    Tc, rc = critical_point(a, b, R)
    if T >= Tc:
        raise ValueError("no spinodal above T_c")
    f = lambda r: dp0_drho(r, T, a, b, R)
    r_g = optimize.brentq(f, 1e-300, rc, xtol=1e-300, rtol=1e-15)
    r_l = optimize.brentq(f, rc, 4.0 / b * (1 - 1e-12), xtol=1e-300, rtol=1e-15)
    return r_g, r_l


def _gas_branch(P, T, r_sp, a, b, R):
    """Density on the gas branch (0, r_sp) with p0 = P, solved in log rho."""
    g = lambda s: p0(math.exp(s), T, a, b, R) - P
    return math.exp(optimize.brentq(g, math.log(1e-300), math.log(r_sp),
                                    xtol=1e-15, rtol=1e-15))


def _liq_branch(P, T, r_sp, a, b, R):
    g = lambda r: p0(r, T, a, b, R) - P
    return optimize.brentq(g, r_sp, 4.0 / b * (1 - 1e-14), xtol=1e-300, rtol=1e-15)


def maxwell(T_r, a=A_CS, b=B_CS, R=R_CS):
    """Maxwell coexistence densities (rho_g, rho_l) at reduced temperature T_r:
    equal pressure on the two stable branches and equal chemical potential,
    found by bisection on the saturation pressure (Sec. 5.1)."""
    Tc, _ = critical_point(a, b, R)
    T = T_r * Tc
    r_sg, r_sl = spinodals(T, a, b, R)
    P_hi = p0(r_sg, T, a, b, R)
    P_lo = max(p0(r_sl, T, a, b, R), 0.0)

    def dmu(logP):
        P = math.exp(logP)
        rg = _gas_branch(P, T, r_sg, a, b, R)
        rl = _liq_branch(P, T, r_sl, a, b, R)
        return mu0(rg, T, a, b, R) - mu0(rl, T, a, b, R)
    lo = math.log(P_lo) if P_lo > 0 else math.log(P_hi) - 600.0
    hi = math.log(P_hi)
    # shrink the bracket ends slightly inside the branches
    logP = optimize.brentq(dmu, lo + 1e-12, hi - 1e-12, xtol=1e-15, rtol=1e-15)
    P = math.exp(logP)
    return _gas_branch(P, T, r_sg, a, b, R), _liq_branch(P, T, r_sl, a, b, R)


def omega(rho, T, rho_b, a=A_CS, b=B_CS, R=R_CS):
    """psi(rho) - psi(rho_b) - mu_b (rho - rho_b), the right side of Eq. 22, with
    psi from Eq. 9: equals rho (mu0(rho) - mu_b) - (p0(rho) - p0(rho_b))."""
    mu_b = mu0(rho_b, T, a, b, R)
    return rho * (mu0(rho, T, a, b, R) - mu_b) - (p0(rho, T, a, b, R) - p0(rho_b, T, a, b, R))


def flat_gradient(rho, T, rho_b, kappa, k, a=A_CS, b=B_CS, R=R_CS):
    """|d rho / d y-hat| of Eq. 24 in the mesh space: the bulk free energy is
    scaled by k^2 (Eq. 28) and kappa is the mesh-space kappa-hat (Eq. 33), so
    (kappa/2)(d rho/dy)^2 = k^2 Omega(rho)."""
    om = np.maximum(omega(rho, T, rho_b, a, b, R), 0.0)
    return np.sqrt(2.0 * k * k * om / kappa)


def flat_profile_y(rho_values, T_r, kappa, k, a=A_CS, b=B_CS, R=R_CS):
    """Mesh-space coordinate y(rho) of the flat interface, Eq. 23, with the origin
    at rho = (rho_g + rho_l)/2 and y increasing towards the liquid.  This is the
    continuum profile for the given kappa; the lattice scheme's own equilibrium
    has kappa + c_s^4/(4 rho) in its place (the exact-difference forcing's
    momentum flux at rest), which tests/test_oracle_physics.py derives and
    checks."""
    Tc, _ = critical_point(a, b, R)
    T = T_r * Tc
    rg, rl = maxwell(T_r, a, b, R)
    r0 = 0.5 * (rg + rl)
    out = []
    for r in np.atleast_1d(rho_values):
        if not (rg < r < rl):
            raise ValueError("density outside (rho_g, rho_l)")
        integrand = lambda s: 1.0 / flat_gradient(s, T, rl, kappa, k, a, b, R)
        val, _ = integrate.quad(integrand, r0, r, limit=400, epsabs=0, epsrel=1e-11)
        out.append(val)
    return np.array(out)


def sigma_flat(T_r, kappa, k, a=A_CS, b=B_CS, R=R_CS):
    """Mesh-space surface tension of the flat interface: the integral of
    P_N - P_T = kappa (d rho/dy)^2 across the interface (Eq. 10), which by
    Eq. 24 becomes the integral of sqrt(2 kappa k^2 Omega(rho)) d rho.  The
    tension the lattice scheme realises has kappa + c_s^4/(4 rho) in place of
    kappa inside the root; tests/test_oracle_physics.py integrates that form."""
    Tc, _ = critical_point(a, b, R)
    T = T_r * Tc
    rg, rl = maxwell(T_r, a, b, R)
    f = lambda r: math.sqrt(max(2.0 * kappa * k * k * float(omega(r, T, rl, a, b, R)), 0.0))
    pts = np.geomspace(rg, rl, 12)[1:-1]
    val, _ = integrate.quad(f, rg, rl, points=pts, limit=400, epsabs=0, epsrel=1e-11)
    return val


def laplace_pair(T_r, kappa, k, radius, a=A_CS, b=B_CS, R=R_CS):
    """Bulk densities (rho_out, rho_in) of a liquid drop of radius `radius` (mesh
    units): equal chemical potential inside and outside, and a pressure jump
    k^2 [p0(rho_in) - p0(rho_out)] = sigma-hat / radius (Eq. 40, pressures
    moved to the mesh space by Eq. 29)."""
    Tc, _ = critical_point(a, b, R)
    T = T_r * Tc
    rg, rl = maxwell(T_r, a, b, R)
    r_sg, r_sl = spinodals(T, a, b, R)
    target = sigma_flat(T_r, kappa, k, a, b, R) / radius / (k * k)

    def resid(log_rg):
        r_out = math.exp(log_rg)
        m = mu0(r_out, T, a, b, R)
        r_in = optimize.brentq(lambda r: mu0(r, T, a, b, R) - m, r_sl,
                               4.0 / b * (1 - 1e-14), xtol=1e-300, rtol=1e-15)
        return p0(r_in, T, a, b, R) - p0(r_out, T, a, b, R) - target, r_in
    s0 = math.log(rg)
    s1 = min(math.log(r_sg) - 1e-9, s0 + 1.0)
    s = optimize.brentq(lambda s: resid(s)[0], s0, s1, xtol=1e-15, rtol=1e-15)
    return math.exp(s), resid(s)[1]
