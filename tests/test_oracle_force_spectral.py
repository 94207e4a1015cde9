"""The oracle's whole force stage (Eqs. 12, 33 with the compact derivatives of
Eqs. 37-39) against an independent Fourier evaluation, on arbitrary fields.

On a periodic line the compact scheme is a circulant operator: the Fourier mode
exp(i w n) is an eigenvector with eigenvalue i theta(w), theta the scheme's
modified wavenumber (A sin w + B/2 sin 2w) / (1 + 2 alpha cos w).  So D u is
ifft(i theta fft(u)), a different computation from the oracle's cyclic
tridiagonal solve.  With walls in y every y-line is first extended evenly about
both walls (period 2 ny) and the same holds on the extended line; the second
y-derivative of the density is the operator applied twice there.

The Fourier evaluation composes mu-hat = k^2 mu0(rho) - kappa-hat (D_x D_x rho +
D_yy rho) and F = -rho D mu-hat + c_s^2 D rho from numpy's mu0 (pinned by
Gibbs-Duhem and the closed-form critical constants).  It is compared on a noisy
drop of unequal sides, periodic and with walls, for CS and PR, both orders: a
dropped or sign-flipped term, x and y exchanged, the Laplacian's second
derivative taken along the wrong axis or a mu-hat extended oddly at a wall fails.
"""
import numpy as np
import pytest

from oracle import OracleSim, cfd_alpha
from oracle import eos as E
from paper_1906_09530_gb300 import workloads as W


def theta(alpha, w):
    A = 2.0 / 3.0 * (alpha + 2.0)
    B = (4.0 * alpha - 1.0) / 3.0
    return (A * np.sin(w) + B / 2 * np.sin(2 * w)) / (1 + 2 * alpha * np.cos(w))


def spectral_d(u, axis, alpha, times=1, even=False):
    """The compact derivative applied `times` times along `axis` by its Fourier
    symbol; `even`: on the line extended evenly about both ends."""
    u = np.moveaxis(u, axis, -1)
    n = u.shape[-1]
    if even:
        u = np.concatenate([u, u[..., ::-1]], axis=-1)
    sym = (1j * theta(alpha, 2 * np.pi * np.fft.fftfreq(u.shape[-1]))) ** times
    d = np.fft.ifft(sym * np.fft.fft(u, axis=-1), axis=-1).real[..., :n]
    return np.moveaxis(d, -1, axis)


def fourier_force_stage(rho, eos, T, kappa, k, alpha, walls):
    dx = lambda u, m=1: spectral_d(u, 1, alpha, m)  # noqa: E731
    dy = lambda u, m=1: spectral_d(u, 0, alpha, m, even=walls)  # noqa: E731
    mu = k * k * eos.mu0(rho, T) - kappa * (dx(dx(rho)) + dy(rho, 2))
    return mu, -rho * dx(mu) + dx(rho) / 3, -rho * dy(mu) + dy(rho) / 3


@pytest.mark.parametrize("kind,omega", [("cs", 0.0), ("pr", 0.344)])
@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("walls", [False, True])
def test_force_stage_equals_fourier_evaluation(kind, omega, order, walls):
    nx, ny, t_r, kappa, k = 40, 28, 0.7, 0.07, 0.4
    eos = E.Eos(kind, omega=omega)
    T = t_r * eos.critical_point()[0]
    rg, rl = eos.maxwell(t_r)
    rho = W.with_noise(W.drop(nx, ny, rg, rl, 7.5, 3.0), 11, 1e-2)
    s = OracleSim(nx, ny, T, kappa, 1.0, k, order, eos=eos, walls_y=walls)
    got = s.force_stage(rho)
    want = fourier_force_stage(rho, eos, T, kappa, k, cfd_alpha(order), walls)
    for g, w in zip(got, want):
        assert np.abs(g - w).max() <= 1e-12 * np.abs(w).max()


def test_fourier_check_sees_the_gradient_term():
    """The comparison above is sensitive to kappa-hat's term: leaving it out of
    the Fourier side moves mu-hat far beyond the tolerance."""
    eos = E.Eos("cs")
    T = 0.7 * eos.critical_point()[0]
    rg, rl = eos.maxwell(0.7)
    rho = W.drop(40, 28, rg, rl, 7.5, 3.0)
    s = OracleSim(40, 28, T, 0.07, 1.0, 0.4, 6, eos=eos)
    mu = s.force_stage(rho)[0]
    bare = fourier_force_stage(rho, eos, T, 0.0, 0.4, cfd_alpha(6), False)[0]
    assert np.abs(mu - bare).max() > 1e-4 * np.abs(mu).max()
