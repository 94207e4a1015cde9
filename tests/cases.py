"""Seeded test cases shared by the GPU parity tests.

The workloads (paper_1906_09530_gb300.workloads) lay out the fields; the
coexistence densities they are built from come from the oracle's thermodynamics,
so no input of a parity test is produced by the CUDA path.

kappa-hat = 0.1 everywhere: the paper does not print kappa, and larger values
(1.0, 0.3) make the k = 1 and k = 0.5 cases blow up in the oracle within 50 steps.
"""
import math

from oracle import thermo
from paper_1906_09530_gb300 import workloads as W

KAPPA = 0.1
TC, RHOC = thermo.critical_point()


def config1(n=128, seed=1234):
    """128^2 static drop, r0 = 24, T_r = 0.7, tanh width 4, k = 1, tau = 1, 4th-order
    compact FD, multiplicative noise 1e-6 (seed 1234)."""
    rg, rl = thermo.maxwell(0.7)
    rho = W.with_noise(W.drop(n, n, rg, rl, 24 * n / 128, 4.0), seed, 1e-6)
    return dict(nx=n, ny=n, T_r=0.7, kappa=KAPPA, tau=1.0, k=1.0, order=4, rho=rho)


def config2(T_r=0.5, n=1024):
    """1024^2 static drop, r0 = 200, k = 0.5, 6th-order compact FD, tanh width
    W = 4/k = 8, tau = 1, no noise."""
    rg, rl = thermo.maxwell(T_r)
    rho = W.drop(n, n, rg, rl, 200 * n / 1024, 8.0)
    return dict(nx=n, ny=n, T_r=T_r, kappa=KAPPA, tau=1.0, k=0.5, order=6, rho=rho)


def ragged(nx=37, ny=29, T_r=0.6, order=6, ux=0.0):
    """A drop on a grid that is not a multiple of any tile or segment size."""
    rg, rl = thermo.maxwell(T_r)
    rho = W.with_noise(W.drop(nx, ny, rg, rl, 8.0, 4.0), 99, 1e-4)
    return dict(nx=nx, ny=ny, T_r=T_r, kappa=KAPPA, tau=0.9, k=0.5, order=order, rho=rho)


def oracle_sim(c, **kw):
    from oracle import OracleSim
    s = OracleSim(c["nx"], c["ny"], c["T_r"] * TC, c["kappa"], c["tau"], c["k"], c["order"],
                  **kw)
    return s


def gpu_sim(c, precision="fp64", **kw):
    from paper_1906_09530_gb300 import Simulation
    return Simulation(c["nx"], c["ny"], c["T_r"], c["kappa"], c["tau"], c["k"],
                      fd_order=c["order"], precision=precision, **kw)


def rel_err(a, b):
    import numpy as np
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def inf():
    return math.inf
