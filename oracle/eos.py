"""Equations of state of the paper beyond Carnahan-Starling, plain FP64 numpy/scipy.

TEST INFRASTRUCTURE ONLY (part of the oracle): only the tests, the smoke check
and the benchmark's CPU legs use it.  Shares no code with the CUDA library.

Each EOS is written as printed in Sec. 3.2, in mesh-free units (T absolute):
  * VDW   p0 Eq. 14, mu0 Eq. 15
  * RK    p0 Eq. 16 with alpha(T) = 1/sqrt(T), mu0 Eq. 17
  * RKS   p0 Eq. 16 with the Soave alpha(T_r) and acentric factor omega, mu0 Eq. 17
  * PR    p0 Eq. 18 with the PR alpha(T_r) and omega, mu0 Eq. 19
  * CS    p0 Eq. 20, mu0 Eq. 21
(mu0 is the chemical potential without its gradient term.)  The paper's
parameters (Sec. 3.2): a = 9/49, b = 2/21 for VDW; a = 2/49, b = 2/21 for RK,
RKS and PR; a = 1, b = 4 for CS; R = 1; omega = 0.344 (water) or 0.011 (methane).

Derived quantities, from their definitions:
  * the critical point: the top of the spinodal curve dp0/drho = 0 (T_r = T/T_c),
    with alpha(T_c) = 1 for RKS and PR (their alpha is defined through T_r) and
    alpha = 1/sqrt(T) inside the spinodal condition for RK;
  * Maxwell coexistence: equal pressure and equal chemical potential (Sec. 5.1).
"""
import math

import numpy as np
from scipy import optimize

KINDS = ("cs", "vdw", "rk", "rks", "pr")
PAPER_AB = {"cs": (1.0, 4.0), "vdw": (9.0 / 49.0, 2.0 / 21.0), "rk": (2.0 / 49.0, 2.0 / 21.0),
            "rks": (2.0 / 49.0, 2.0 / 21.0), "pr": (2.0 / 49.0, 2.0 / 21.0)}
SQ2 = math.sqrt(2.0)


class Eos:
    def __init__(self, kind, a=None, b=None, R=1.0, omega=0.0):
        if kind not in KINDS:
            raise ValueError(kind)
        self.kind = kind
        a0, b0 = PAPER_AB[kind]
        self.a = a0 if a is None else a
        self.b = b0 if b is None else b
        self.R = R
        self.omega = omega
        self._tc = None

    # ---- temperature functions (Sec. 3.2) --------------------------------
    def alpha(self, T):
        """alpha(T) of Eqs. 16-19 (1 for VDW and CS)."""
        if self.kind == "rk":
            return 1.0 / math.sqrt(T)
        if self.kind in ("rks", "pr"):
            w = self.omega
            if self.kind == "rks":
                m = 0.480 + 1.574 * w - 0.176 * w * w
            else:
                m = 0.37464 + 1.54226 * w - 0.26992 * w * w
            return (1.0 + m * (1.0 - math.sqrt(T / self.critical_point()[0]))) ** 2
        return 1.0

    @property
    def rho_max(self):
        """The repulsive pole: b rho = 1 (cubic EOSs), b rho / 4 = 1 (CS)."""
        return 4.0 / self.b if self.kind == "cs" else 1.0 / self.b

    # ---- p0 and mu0 as printed --------------------------------------------
    def p0(self, rho, T, alpha=None):
        a, b, R = self.a, self.b, self.R
        al = self.alpha(T) if alpha is None else alpha
        if self.kind == "cs":  # Eq. 20
            e = b * rho / 4.0
            return rho * R * T * (1 + e + e**2 - e**3) / (1 - e) ** 3 - a * rho**2
        rep = rho * R * T / (1 - b * rho)
        if self.kind == "vdw":  # Eq. 14
            return rep - a * rho**2
        if self.kind in ("rk", "rks"):  # Eq. 16
            return rep - a * al * rho**2 / (1 + b * rho)
        return rep - a * al * rho**2 / (1 + 2 * b * rho - b**2 * rho**2)  # Eq. 18

    def mu0(self, rho, T, alpha=None):
        a, b, R = self.a, self.b, self.R
        al = self.alpha(T) if alpha is None else alpha
        if self.kind == "cs":  # Eq. 21
            e = b * rho / 4.0
            return R * T * ((3 - e) / (1 - e) ** 3 + np.log(rho) + 1) - 2 * a * rho
        if self.kind == "vdw":  # Eq. 15
            return R * T * (np.log(rho / (1 - b * rho)) + 1 / (1 - b * rho)) - 2 * a * rho
        if self.kind in ("rk", "rks"):  # Eq. 17
            return (R * T * np.log(rho / (1 - b * rho)) + R * T / (1 - b * rho)
                    - a * al / b * np.log(1 + b * rho) - a * al * rho / (1 + b * rho))
        return (R * T * np.log(rho / (1 - b * rho))  # Eq. 19
                - a * al / (2 * SQ2 * b) * np.log((SQ2 - 1 + b * rho) / (SQ2 + 1 - b * rho))
                + R * T / (1 - b * rho) - a * al * rho / (1 + 2 * b * rho - b**2 * rho**2))

    def dp0_drho(self, rho, T, alpha=None):
        """d p0 / d rho by the complex-step derivative (exact to rounding for
        these analytic p0)."""
        h = 1e-30
        return (self.p0(rho + 1j * h, T, alpha)).imag / h

    # ---- critical point -----------------------------------------------------
    def _spinodal_T(self, rho):
        """The temperature at which dp0/drho = 0 at this density (alpha at
        criticality: 1 for RKS/PR, 1/sqrt(T) for RK)."""
        def f(T):
            al = 1.0 / math.sqrt(T) if self.kind == "rk" else 1.0
            return self.dp0_drho(rho, T, al)
        lo, hi = 1e-12, 1.0
        while f(hi) < 0:
            hi *= 2.0
        return optimize.brentq(f, lo, hi, xtol=1e-300, rtol=1e-15, maxiter=500)

    def critical_point(self):
        """(T_c, rho_c): the maximum of the spinodal temperature over density."""
        if self._tc is None:
            rmax = self.rho_max
            res = optimize.minimize_scalar(lambda r: -self._spinodal_T(r),
                                           bounds=(0.02 * rmax, 0.9 * rmax), method="bounded",
                                           options={"xatol": 1e-13 * rmax, "maxiter": 500})
            self._tc = (-res.fun, res.x)
        return self._tc

    # ---- Maxwell coexistence ------------------------------------------------
    def spinodals(self, T):
        """Densities where dp0/drho = 0 at T < T_c (gas side, liquid side)."""
        tc, rc = self.critical_point()
        al = self.alpha(T)
        f = lambda r: self.dp0_drho(r, T, al)
        sg = optimize.brentq(f, 1e-300, rc, xtol=1e-300, rtol=1e-15, maxiter=2000)
        sl = optimize.brentq(f, rc, self.rho_max * (1 - 1e-14), xtol=1e-300, rtol=1e-15,
                             maxiter=2000)
        return sg, sl

    def maxwell(self, T_r):
        """(rho_g, rho_l) at T = T_r T_c: equal p0 and equal mu0 on the two
        branches, found by brentq on the logarithm of the saturation pressure,
        bracketed by the spinodal pressures."""
        tc, _ = self.critical_point()
        T = T_r * tc
        al = self.alpha(T)
        sg, sl = self.spinodals(T)

        def gas(P):  # on (0, sg), solved in log rho
            g = lambda s: self.p0(math.exp(s), T, al) - P
            return math.exp(optimize.brentq(g, math.log(1e-300), math.log(sg), xtol=1e-15,
                                            rtol=1e-15, maxiter=2000))

        def liq(P):
            g = lambda r: self.p0(r, T, al) - P
            return optimize.brentq(g, sl, self.rho_max * (1 - 1e-14), xtol=1e-300, rtol=1e-15,
                                   maxiter=2000)

        def dmu(logP):
            P = math.exp(logP)
            return self.mu0(gas(P), T, al) - self.mu0(liq(P), T, al)

        p_hi = self.p0(sg, T, al)
        p_lo = max(self.p0(sl, T, al), 0.0)
        lo = math.log(p_lo) if p_lo > 0 else math.log(p_hi) - 600.0
        hi = math.log(p_hi)
        logP = optimize.brentq(dmu, lo + 1e-12, hi - 1e-12, xtol=1e-15, rtol=1e-15,
                               maxiter=500)
        P = math.exp(logP)
        return gas(P), liq(P)
