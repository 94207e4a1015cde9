"""The equilibrium of a flat periodic interface, found directly as the fixed point
of the scheme's time step.

TEST INFRASTRUCTURE ONLY (part of the oracle): only the tests and the
benchmark's CPU legs use it.  Shares no code with the CUDA library, and no code
with the C oracle either: it restates the same time step in numpy, which the
tests check against the C oracle's own time stepping.

A slab uniform along x is a 1-D problem along y.  With u_x = 0 and the
populations of e_x = +1 and e_x = -1 equal, the nine D2Q9 populations of a node
reduce to six values (velocity order of Sec. 2):
  g0 = f0, gx = f1 = f3, gu = f2, gd = f4, gux = f5 = f6, gdx = f7 = f8,
with multiplicities (1, 2, 1, 1, 2, 2) in the moments of Eq. 3.  One time step,
in the order the method is run (the force from the density of the populations
before the collision):
  * the force stage, Eqs. 12, 33, 37-39: mu-hat = k^2 mu0(rho) - kappa D(D rho),
    F = -rho D mu-hat + c_s^2 D rho, with D the periodic compact derivative;
  * exact-difference forcing and BGK collision, Eqs. 1, 2, 5:
    g* = g - (g - g^eq(rho, u)) / tau + g^eq(rho, u + F/rho) - g^eq(rho, u);
  * streaming along y (Eq. 1): populations with e_y = +1 move up one node,
    e_y = -1 down one, periodically.
That step is a map g -> M(g) of the 6 n values.  A run relaxes to the fixed
point of M with the run's mass; it is found here by Newton's method on
M(g) - g = 0, one equation replaced by the mass.  The Jacobian is taken by the
complex step, exact to rounding because every operation of M is analytic
(the chemical potential's log included).  The C oracle supplies the start: it
runs the slab until the fast transients have died, and Newton removes the slow
diffusive remainder.
"""
import math

import numpy as np

from . import sim
from .eos import Eos

CS2 = 1.0 / 3.0
# per reduced population: weight of Eq. 2, multiplicity, e_y
W6 = np.array([4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0, 1.0 / 36.0])
MULT = np.array([1.0, 2.0, 1.0, 1.0, 2.0, 2.0])
EY6 = np.array([0.0, 0.0, 1.0, -1.0, 1.0, -1.0])


def cfd_matrix(n, order):
    """Dense matrix of the periodic compact first derivative on n points,
    Eqs. 37-38 with h = 1: D = A^-1 B, (A d)_i = alpha d_{i-1} + d_i +
    alpha d_{i+1}, (B u)_i = a (u_{i+1} - u_{i-1})/2 + b (u_{i+2} - u_{i-2})/4."""
    alpha = sim.cfd_alpha(order)
    a = 2.0 / 3.0 * (alpha + 2.0)
    b = (4.0 * alpha - 1.0) / 3.0
    A = np.zeros((n, n))
    B = np.zeros((n, n))
    for i in range(n):
        A[i, i] = 1.0
        A[i, (i - 1) % n] += alpha
        A[i, (i + 1) % n] += alpha
        B[i, (i + 1) % n] += a / 2.0
        B[i, (i - 1) % n] -= a / 2.0
        B[i, (i + 2) % n] += b / 4.0
        B[i, (i - 2) % n] -= b / 4.0
    return np.linalg.solve(A, B)


class FlatSlab:
    """The scheme on a periodic line of n nodes along y, BGK with relaxation
    time tau, equation of state `eos` (an oracle.eos.Eos; Carnahan-Starling
    with a = 1, b = 4, R = 1 when None) at reduced temperature T_r."""

    # Readings of the paper other than the one the method is run with, kept to
    # audit it (each changes one step; "printed" is the method):
    #   "cs2_mesh"       c_s^2 of Eq. 12 taken as the mesh-space k^2 c_s^2 (Eq. 26)
    #   "ideal_central"  the c_s^2 grad rho of Eq. 12 by the central difference
    #                    of Eq. 34 instead of the compact scheme
    #   "collide_to_v"   the collision of Eq. 1 towards f^eq(rho, v), v the
    #                    redefined velocity u + F/(2 rho) of Sec. 2
    #   "forcing_at_v"   the increment of Eq. 5 taken about v instead of u
    READINGS = ("printed", "cs2_mesh", "ideal_central", "collide_to_v", "forcing_at_v")

    def __init__(self, n, T_r, kappa, tau, k, order=6, eos=None, reading="printed"):
        if reading not in self.READINGS:
            raise ValueError(reading)
        self.reading = reading
        self.n, self.kappa, self.tau, self.k, self.order = n, kappa, tau, k, order
        self.eos = eos if eos is not None else Eos("cs")
        Tc, _ = self.eos.critical_point()
        self.T_r = T_r
        self.T = T_r * Tc
        self.al = self.eos.alpha(self.T)
        self.D = cfd_matrix(n, order)

    # ---- the time step -------------------------------------------------
    def moments(self, g):
        """rho and rho u_y of states g [6, n, ...]."""
        m = MULT.reshape((6,) + (1,) * (g.ndim - 1))
        e = EY6.reshape(m.shape)
        return (m * g).sum(0), (m * e * g).sum(0)

    def feq(self, rho, u):
        w = W6.reshape((6,) + (1,) * rho.ndim)
        e = EY6.reshape(w.shape)
        eu = e * u
        return w * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * u * u)

    def force(self, rho):
        """(mu-hat, F_y) of a density [n, ...] (Eqs. 12 and 33)."""
        d_rho = self.D @ rho
        mu = self.k ** 2 * self.eos.mu0(rho, self.T, self.al) - self.kappa * (self.D @ d_rho)
        if self.reading == "cs2_mesh":
            return mu, -rho * (self.D @ mu) + self.k ** 2 * CS2 * d_rho
        if self.reading == "ideal_central":
            return mu, -rho * (self.D @ mu) + CS2 * 0.5 * (np.roll(rho, -1, axis=0)
                                                          - np.roll(rho, 1, axis=0))
        return mu, -rho * (self.D @ mu) + CS2 * d_rho

    def step(self, g):
        """One time step M(g) of states g [6, n] or a batch [6, n, m]."""
        rho, j = self.moments(g)
        u = j / rho
        _, F = self.force(rho)
        feq = self.feq(rho, u)
        if self.reading == "collide_to_v":
            v = u + 0.5 * F / rho
            post = g - (g - self.feq(rho, v)) / self.tau + self.feq(rho, u + F / rho) - feq
        elif self.reading == "forcing_at_v":
            v = u + 0.5 * F / rho
            post = g - (g - feq) / self.tau + self.feq(rho, v + F / rho) - self.feq(rho, v)
        else:
            post = g - (g - feq) / self.tau + self.feq(rho, u + F / rho) - feq
        out = np.empty_like(post)
        out[0:2] = post[0:2]
        out[2] = np.roll(post[2], 1, axis=0)   # e_y = +1 arrives from the node below
        out[4] = np.roll(post[4], 1, axis=0)
        out[3] = np.roll(post[3], -1, axis=0)  # e_y = -1 from the node above
        out[5] = np.roll(post[5], -1, axis=0)
        return out

    # ---- states ----------------------------------------------------------
    def from_populations(self, f):
        """The reduced state of 2-D populations f[9][ny][nx] that are uniform in
        x, taken from column 0."""
        c = f[:, :, 0]
        return np.array([c[0], c[1], c[2], c[4], c[5], c[7]])

    def fields(self, g):
        """(rho, v_y, mu-hat, F_y): v = u + F/(2 rho), the velocity of Sec. 2."""
        rho, j = self.moments(g)
        mu, F = self.force(rho)
        return rho, (j + 0.5 * F) / rho, mu, F

    # ---- the fixed point ---------------------------------------------------
    def residual(self, g):
        return (self.step(g) - g).reshape(-1)

    def jacobian(self, g, h=1e-30, directions=None):
        """(d M(g) / d g - I) V, by the complex step, for the columns of V
        (`directions`, [6n, m]; the identity when None: the full [6n, 6n])."""
        N = g.size
        V = np.eye(N) if directions is None else directions
        G = g.reshape(-1, 1).astype(np.complex128) + 1j * h * V
        Mg = self.step(G.reshape((6, self.n, V.shape[1])))
        return Mg.reshape(N, V.shape[1]).imag / h - V

    def symmetric_basis(self):
        """(P, rows): states that are even about node 0 (and so about node n/2),
        g = P s, and the residual rows that are independent on such states.
        The mirror y -> -y keeps g0 and gx and swaps gu <-> gd, gux <-> gdx.
        Restricting Newton to these states removes the slab's near-translation
        (a singular value about 1e-11 of the full Jacobian)."""
        n, h = self.n, self.n // 2
        cols = []
        P = np.zeros((6 * n, 2 * (h + 1) + 2 * n))
        c = 0
        for q in (0, 1):  # g0, gx: even
            for j in range(h + 1):
                P[q * n + j, c] = 1.0
                P[q * n + (-j) % n, c] = 1.0
                c += 1
        for up, dn in ((2, 3), (4, 5)):  # gu(j) = gd(-j), gux(j) = gdx(-j)
            for j in range(n):
                P[up * n + j, c] = 1.0
                P[dn * n + (-j) % n, c] = 1.0
                c += 1
        rows = [q * n + j for q in (0, 1) for j in range(h + 1)] + \
            [q * n + j for q in (2, 4) for j in range(n)]
        return P, np.array(rows)

    def relative_residual(self, g):
        """Largest residual of the fixed-point equations relative to its own
        component (the gas populations are up to 1e14 times the liquid's)."""
        return float(np.max(np.abs(self.residual(g)) / np.abs(g.reshape(-1))))

    def newton(self, g, tol=1e-13, max_iter=40):
        """The fixed point with g's mass, from the start g (made even about node
        0 first); returns (g, largest residual relative to the largest
        population, iterations).  Below T_r ~ 0.25 that measure leaves the
        dilute gas unresolved (its populations are 1e9 and more times smaller):
        flat_equilibrium then finishes by time stepping (polish)."""
        n = self.n
        P, rows = self.symmetric_basis()
        g = np.array(g, dtype=np.float64)
        mrow = np.repeat(MULT, n)
        mass0 = float(mrow @ g.reshape(-1))
        # the even part of the start: average it with its mirror image
        s = np.linalg.lstsq(P, g.reshape(-1), rcond=None)[0]
        g = (P @ s).reshape(6, n)
        g *= mass0 / float(mrow @ g.reshape(-1))
        s = np.linalg.lstsq(P, g.reshape(-1), rcond=None)[0]
        mP = mrow @ P
        res = np.inf
        for it in range(1, max_iter + 1):
            g = (P @ s).reshape(6, n)
            r_full = self.residual(g)
            A = self.jacobian(g, directions=P)[rows]
            r = r_full[rows]
            A[0, :] = mP  # one equation is redundant (mass is conserved): use the mass
            r[0] = float(mP @ s) - mass0
            ds = np.linalg.solve(A, -r)
            # damped step: halve it until the density stays positive and the
            # residual does not grow (full steps once close)
            r_now = float(np.abs(r_full).max())
            lam = 1.0
            while True:
                trial = s + lam * ds
                gt = (P @ trial).reshape(6, n)
                if self.moments(gt)[0].min() > 0:
                    r_try = float(np.abs(self.residual(gt)).max())
                    if np.isfinite(r_try) and (r_try < r_now or lam < 1e-3):
                        break
                lam *= 0.5
                if lam < 1e-6:
                    return g, r_now / np.abs(g).max(), it
            s = trial
            g = gt
            res = r_try / float(np.abs(g).max())
            if res < tol and lam * float(np.abs(ds).max()) < 1e3 * tol * float(np.abs(s).max()):
                return g, res, it
        return g, res, max_iter

    def polish(self, g, block=10000, max_blocks=60, rtol=1e-9):
        """Advance the state g with the C oracle (nx = 8, uniform in x) in blocks
        of `block` steps until the density at every node changes by less than
        rtol (relative) over a block; returns (g, steps taken)."""
        f = np.zeros((9, self.n, 8))
        for i, q in enumerate((0, 1, 2, 1, 3, 4, 4, 5, 5)):
            f[i] = g[q][:, None]
        o = sim.OracleSim(8, self.n, self.T, self.kappa, self.tau, self.k, self.order,
                          eos=self.eos)
        o.set_populations(f, 0)
        prev = self.moments(g)[0]
        for _ in range(max_blocks):
            o.step(block)
            cur = o.fields()[0][:, 0]
            done = float(np.max(np.abs(cur / prev - 1))) < rtol
            prev = cur
            if done:
                break
        return self.from_populations(o.f), o.t


def slab_start(n, T_r, kappa, tau, k, order=6, eos=None, steps=20000, width=None):
    """Populations of a slab between the Maxwell densities (a tanh of width 4/k
    about each interface, the liquid in the middle half of the line), advanced
    `steps` steps by the C oracle (nx = 8, uniform in x)."""
    e = eos if eos is not None else Eos("cs")
    rg, rl = e.maxwell(T_r)
    w = 4.0 / k if width is None else width
    y = np.arange(n, dtype=np.float64)[:, None] * np.ones((1, 8))
    d = np.abs(y - n / 2.0) - n / 4.0
    rho = 0.5 * (rg + rl) + 0.5 * (rg - rl) * np.tanh(2.0 * d / w)
    Tc, _ = e.critical_point()
    o = sim.OracleSim(8, n, T_r * Tc, kappa, tau, k, order, eos=eos)
    o.set_fields(rho)
    if steps:
        o.step(steps)
    return o.f, (rg, rl)


def flat_equilibrium(n, T_r, kappa, tau, k, order=6, eos=None, steps=20000, reading="printed"):
    """The converged flat slab: dict with the profile and the bulk densities
    (the gas at the node farthest from both interfaces, the liquid at the slab's
    centre), their offsets from Maxwell, and the Newton residual."""
    slab = FlatSlab(n, T_r, kappa, tau, k, order, eos, reading)
    if reading == "printed":
        f, (rg, rl) = slab_start(n, T_r, kappa, tau, k, order, eos, steps)
        g = slab.from_populations(f)
    else:  # the C oracle runs the printed method only: step this reading here
        f, (rg, rl) = slab_start(n, T_r, kappa, tau, k, order, eos, 0)
        g = slab.from_populations(f)
        for _ in range(steps):
            g = slab.step(g)
    g_start = g
    g, res, it = slab.newton(g)
    polished = 0
    if reading == "printed" and slab.relative_residual(g) > 1e-10:
        # Newton's state is the start of the polish when it has the gas nearly
        # right; when it does not (relative residual above 1e-6, below T_r ~ 0.2),
        # the time-stepped start is, as a wrong dilute gas can drive the run
        # unstable
        if slab.relative_residual(g) > 1e-6:
            g, polished = slab.polish(g_start, max_blocks=300)
        else:
            g, polished = slab.polish(g)
    rho, v, mu, F = slab.fields(g)
    gas, liq = float(rho[0]), float(rho[n // 2])
    return {"rho": rho, "v": v, "mu": mu, "F": F, "g": g, "rho_g": gas, "rho_l": liq,
            "maxwell": (rg, rl), "gas_offset": gas / rg - 1.0, "liq_offset": liq / rl - 1.0,
            "log10_gas_offset": math.log10(gas / rg), "residual": res, "iterations": it,
            "relative_residual": slab.relative_residual(g), "polish_steps": polished}
