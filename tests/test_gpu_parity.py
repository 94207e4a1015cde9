"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs.

Tolerances (written here, justified by the arithmetic):
  * compact-FD solves: |d_gpu - d_oracle| <= 1e-13 max|d_oracle|.  Both are FP64;
    the factorised sweep truncates recursions whose tail weight is < 1e-18, so
    only rounding-order differences remain.
  * force stage at t = 0: mu-hat and v = F/(2 rho) within 1e-12 (relative to max).
  * full FP64 steps: pointwise rho relative error <= 1e-10 after 1000 steps
    (the FP64 path's stated tolerance), v and mu-hat within 1e-8 of their max.
  * mixed path: populations in FP32 (unit rounding 6e-8).  Its stated bound is on
    the coexistence densities (within 1e-3 of Maxwell); node by node against the
    FP64 oracle, the 128^2 k = 1 drop (velocities ~0.03, the most dynamic case)
    stays within 1e-4 after 200 steps (measured 4.4e-5).
"""

import numpy as np
import pytest

from tests import cases

pytestmark = pytest.mark.gpu


def rel_point(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("shape", [(8, 8), (37, 50), (128, 96), (1024, 64), (5, 300)])
@pytest.mark.parametrize("axis", [0, 1])
def test_cfd_parity(cuda, order, shape, axis):
    from oracle import cfd_alpha, cfd_line
    from paper_1906_09530_gb300 import lbm_cfd
    torch = cuda
    ny, nx = shape
    rng = np.random.default_rng(nx * 1000 + ny + order)
    u = rng.standard_normal((ny, nx)) + 3.0
    d1, d2 = lbm_cfd(torch.from_numpy(u).cuda(), axis, order, second=True)
    torch.cuda.synchronize()
    d1, d2 = d1.cpu().numpy(), d2.cpu().numpy()
    alpha = cfd_alpha(order)
    if axis == 0:
        r1 = np.stack([cfd_line(u[j], alpha) for j in range(ny)])
    else:
        r1 = np.stack([cfd_line(u[:, i], alpha) for i in range(nx)], axis=1)
    if axis == 0:
        r2 = np.stack([cfd_line(r1[j], alpha) for j in range(ny)])
    else:
        r2 = np.stack([cfd_line(r1[:, i], alpha) for i in range(nx)], axis=1)
    assert np.abs(d1 - r1).max() <= 1e-13 * np.abs(r1).max()
    assert np.abs(d2 - r2).max() <= 1e-13 * np.abs(r2).max()
    # first derivative alone (the single-recursion kernel)
    d1b = lbm_cfd(torch.from_numpy(u).cuda(), axis, order, second=False).cpu().numpy()
    assert np.abs(d1b - r1).max() <= 1e-13 * np.abs(r1).max()


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("shape", [(8, 8), (37, 50), (96, 128), (64, 1024), (300, 5)])
@pytest.mark.parametrize("axis", [0, 1])
def test_cfd_df_parity(cuda, order, shape, axis):
    """The mixed path's double-float line solve on a field with a liquid/gas
    dynamic range of 1e8: first derivative within 1e-13 of the line maximum plus
    FP32 rounding of the result itself; second derivative (FP32) within 1e-6 of
    its maximum."""
    from oracle import cfd_alpha, cfd_line
    from paper_1906_09530_gb300 import lbm_cfd_df
    torch = cuda
    ny, nx = shape
    rng = np.random.default_rng(nx * 7 + ny + order)
    u = 1e-8 * (1 + 0.1 * rng.standard_normal((ny, nx)))
    if axis == 0:
        u[:, nx // 3: 2 * nx // 3] = 0.5 + 0.01 * rng.standard_normal((ny, 2 * nx // 3 - nx // 3))
    else:
        u[ny // 3: 2 * ny // 3, :] = 0.5 + 0.01 * rng.standard_normal((2 * ny // 3 - ny // 3, nx))
    hi = u.astype(np.float32)
    lo = (u - hi.astype(np.float64)).astype(np.float32)
    uu = hi.astype(np.float64) + lo.astype(np.float64)
    d1, d2 = lbm_cfd_df(torch.from_numpy(hi).cuda(), torch.from_numpy(lo).cuda(), axis, order,
                        second=True)
    d1 = d1.cpu().numpy().astype(np.float64)
    d2 = d2.cpu().numpy().astype(np.float64)
    alpha = cfd_alpha(order)
    lines = (lambda a: np.stack([cfd_line(a[j], alpha) for j in range(ny)])) if axis == 0 else \
        (lambda a: np.stack([cfd_line(a[:, i], alpha) for i in range(nx)], axis=1))
    r1 = lines(uu)
    r2 = lines(r1)
    tol1 = 1e-13 * np.abs(r1).max() + 2.0 ** -24 * np.abs(r1)
    assert np.all(np.abs(d1 - r1) <= tol1)
    assert np.abs(d2 - r2).max() <= 1e-6 * np.abs(r2).max()


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("axis", [0, 1])
def test_cfd_df_smooth_window_parity(cuda, order, axis):
    """Windows whose staged values span less than a factor 32 are solved in FP32
    (double-float is only needed across an interface): there the result is
    within FP32 rounding of the values along the line (1e-5 of max|u|)."""
    from oracle import cfd_alpha, cfd_line
    from paper_1906_09530_gb300 import lbm_cfd_df
    torch = cuda
    ny, nx = 96, 700
    rng = np.random.default_rng(order + 10 * axis)
    y, x = np.mgrid[0:ny, 0:nx]
    u = 0.3 + 0.1 * np.sin(2 * np.pi * x / nx * 3) * np.cos(2 * np.pi * y / ny * 2) \
        + 1e-3 * rng.standard_normal((ny, nx))
    hi = u.astype(np.float32)
    lo = (u - hi.astype(np.float64)).astype(np.float32)
    uu = hi.astype(np.float64) + lo.astype(np.float64)
    d1, d2 = lbm_cfd_df(torch.from_numpy(hi).cuda(), torch.from_numpy(lo).cuda(), axis, order,
                        second=True)
    d1 = d1.cpu().numpy().astype(np.float64)
    d2 = d2.cpu().numpy().astype(np.float64)
    alpha = cfd_alpha(order)
    lines = (lambda a: np.stack([cfd_line(a[j], alpha) for j in range(ny)])) if axis == 0 else \
        (lambda a: np.stack([cfd_line(a[:, i], alpha) for i in range(nx)], axis=1))
    r1 = lines(uu)
    r2 = lines(r1)
    assert np.abs(d1 - r1).max() <= 1e-5 * np.abs(uu).max()
    assert np.abs(d2 - r2).max() <= 1e-5 * np.abs(uu).max()


@pytest.mark.parametrize("case", ["config1", "ragged4", "ragged6"])
def test_force_stage_parity_t0(cuda, case):
    c = {"config1": cases.config1(), "ragged4": cases.ragged(order=4),
         "ragged6": cases.ragged(order=6)}[case]
    g = cases.gpu_sim(c)
    g.set_fields(c["rho"])
    rho, vx, vy, mu = g.fields()
    o = cases.oracle_sim(c)
    o.set_fields(c["rho"])
    orho, ovx, ovy, omu, _, _ = o.fields()
    assert rel_point(rho, orho) <= 1e-14
    assert cases.rel_err(mu, omu) <= 1e-12
    assert np.abs(vx - ovx).max() <= 1e-12 * np.abs(ovx).max()
    assert np.abs(vy - ovy).max() <= 1e-12 * np.abs(ovy).max()


def test_config1_1000_steps_fp64(cuda):
    """128^2 drop, CS T_r = 0.7, k = 1, 4th order: rho within 1e-10 after 1000 steps."""
    c = cases.config1()
    g = cases.gpu_sim(c)
    g.set_fields(c["rho"])
    g.step(1000)
    rho, vx, vy, mu = g.fields()
    o = cases.oracle_sim(c)
    o.set_fields(c["rho"])
    o.step(1000)
    orho, ovx, ovy, omu, _, _ = o.fields()
    assert g.t == 1000
    assert rel_point(rho, orho) <= 1e-10
    assert np.abs(vx - ovx).max() <= 1e-8 * np.abs(ovx).max()
    assert np.abs(mu - omu).max() <= 1e-8 * np.abs(omu).max()


@pytest.mark.parametrize("order", [4, 6])
def test_ragged_grid_steps(cuda, order):
    """37 x 29: every tile and line segment is ragged; odd step count exercises
    the single-step path after the two-step graphs."""
    c = cases.ragged(order=order)
    g = cases.gpu_sim(c)
    g.set_fields(c["rho"])
    g.step(201)
    o = cases.oracle_sim(c)
    o.set_fields(c["rho"])
    o.step(201)
    assert rel_point(g.fields()[0], o.fields()[0]) <= 1e-11


def test_velocity_init_parity(cuda):
    """Initial velocity (a drop translated at u_x = 0.05, the Galilean variant)."""
    c = cases.ragged(nx=48, ny=40, order=6)
    ux = np.full((40, 48), 0.05)
    uy = np.full((40, 48), -0.02)
    g = cases.gpu_sim(c)
    g.set_fields(c["rho"], ux, uy)
    g.step(100)
    o = cases.oracle_sim(c)
    o.set_fields(c["rho"], ux, uy)
    o.step(100)
    rho, vx, vy, _ = g.fields()
    orho, ovx, ovy, _, _, _ = o.fields()
    assert rel_point(rho, orho) <= 1e-11
    assert np.abs(vx - ovx).max() <= 1e-10


def test_mu_cap_parity(cuda):
    """Sec. 5.6 upper limit active for the first 7 steps."""
    c = cases.ragged(nx=40, ny=40, order=6)
    kw = dict(mu_max=-0.55, mu_cap_steps=7)
    g = cases.gpu_sim(c, **kw)
    g.set_fields(c["rho"])
    o = cases.oracle_sim(c, **kw)
    o.set_fields(c["rho"])
    mu0 = g.fields()[3]
    assert mu0.max() <= 0.25 * -0.55 + 1e-15
    g.step(20)
    o.step(20)
    assert rel_point(g.fields()[0], o.fields()[0]) <= 1e-11


def test_config2_full_size_steps(cuda):
    """1024^2, T_r = 0.5, k = 0.5, 6th order, the launch configuration the benchmark
    times: every node after 4 steps against the oracle."""
    c = cases.config2(0.5)
    g = cases.gpu_sim(c)
    g.set_fields(c["rho"])
    g.step(4)
    o = cases.oracle_sim(c)
    o.set_fields(c["rho"])
    o.step(4)
    assert rel_point(g.fields()[0], o.fields()[0]) <= 1e-12


@pytest.mark.parametrize("precision", ["mixed", "mixed_df"])
def test_config2_mixed_full_size_steps(cuda, precision):
    """1024^2, T_r = 0.45 (ratio 2.3e3: FP32 density lines in "mixed", double-float
    in "mixed_df"), every node after 4 steps against the oracle."""
    c = cases.config2(0.45)
    g = cases.gpu_sim(c, precision=precision)
    g.set_fields(c["rho"])
    g.step(4)
    o = cases.oracle_sim(c)
    o.set_fields(c["rho"])
    o.step(4)
    assert rel_point(g.fields()[0], o.fields()[0]) <= 2e-6


@pytest.mark.parametrize("precision", ["mixed", "mixed_df"])
@pytest.mark.parametrize("case", ["config1", "ragged4", "ragged6"])
def test_mixed_force_stage_t0(cuda, case, precision):
    """Mixed path at t = 0: f^eq rounded to FP32, density kept exactly; mu-hat and
    the force in FP32 against the FP64 oracle."""
    c = {"config1": cases.config1(), "ragged4": cases.ragged(order=4),
         "ragged6": cases.ragged(order=6)}[case]
    g = cases.gpu_sim(c, precision=precision)
    g.set_fields(c["rho"])
    rho, vx, vy, mu = g.fields()
    o = cases.oracle_sim(c)
    o.set_fields(c["rho"])
    orho, ovx, ovy, omu, _, _ = o.fields()
    assert rel_point(rho, orho) <= 2e-7
    assert cases.rel_err(mu, omu) <= 1e-5
    assert np.abs(vx - ovx).max() <= 1e-4 * np.abs(ovx).max()


def test_mixed_close_to_oracle(cuda):
    c = cases.config1()
    g = cases.gpu_sim(c, precision="mixed")
    g.set_fields(c["rho"])
    g.step(200)
    o = cases.oracle_sim(c)
    o.set_fields(c["rho"])
    o.step(200)
    assert rel_point(g.fields()[0], o.fields()[0]) <= 1e-4


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_mass_conservation_large(cuda, precision, tol):
    c = cases.config2(0.5, n=2048)
    g = cases.gpu_sim(c, precision=precision)
    g.set_fields(c["rho"])
    m0 = g.diag()[0]
    assert m0 == pytest.approx(c["rho"].sum(), rel=1e-7 if precision == "mixed" else 1e-13)
    g.step(100)
    assert abs(g.diag()[0] - m0) / m0 <= tol


def test_uniform_rest_fixed_point(cuda):
    from paper_1906_09530_gb300 import Simulation
    g = Simulation(64, 48, 0.6, 0.1, 0.8, 0.5, fd_order=6)
    g.set_fields(np.full((48, 64), 0.25))
    g.step(20)
    rho, vx, vy, mu = g.fields()
    assert np.allclose(rho, 0.25, rtol=1e-14, atol=0)
    assert np.abs(vx).max() < 1e-15 and np.abs(vy).max() < 1e-15


def test_diag_matches_fields(cuda):
    c = cases.ragged(nx=64, ny=64)
    g = cases.gpu_sim(c)
    g.set_fields(c["rho"])
    g.step(10)
    rho, vx, vy, _ = g.fields()
    mass, vmax, rmin, rmax = g.diag()
    assert mass == pytest.approx(rho.sum(), rel=1e-13)
    assert vmax == pytest.approx(np.hypot(vx, vy).max(), rel=1e-12)
    assert (rmin, rmax) == (rho.min(), rho.max())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_checkpoint_resume_bitexact(cuda, precision):
    c = cases.ragged(nx=64, ny=40)
    g = cases.gpu_sim(c, precision=precision)
    g.set_fields(c["rho"])
    g.step(15)
    f, t = g.get_populations()
    assert t == 15
    g.step(11)
    a = g.fields()
    g.set_populations(f, t)
    assert g.t == 15
    g.step(11)
    b = g.fields()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_unstable_is_reported_not_trapped(cuda):
    """A host-written bad density (negative at one node) makes the device raise
    its error flag; the call returns LBM_EUNSTABLE and the context stays usable."""
    from paper_1906_09530_gb300 import LbmError
    from paper_1906_09530_gb300._binding import LBM_EUNSTABLE
    c = cases.ragged(nx=32, ny=32)
    rho = c["rho"].copy()
    rho[5, 7] = -1e-3
    g = cases.gpu_sim(c)
    with pytest.raises(LbmError) as ei:
        g.set_fields(rho)
        g.step(3)
    assert ei.value.status == LBM_EUNSTABLE
    assert 0 <= g.failed_step <= 3
    g.set_fields(c["rho"])  # recovers
    g.step(2)


def test_bounded_wait_reports_timeout(cuda):
    """The host wait has a limit: a tiny limit on a long queue returns
    LBM_ETIMEOUT (the work itself finishes normally afterwards)."""
    from paper_1906_09530_gb300 import LbmError
    from paper_1906_09530_gb300._binding import LBM_ETIMEOUT
    c = cases.config2(0.5, n=1024)
    g = cases.gpu_sim(c)
    g.set_fields(c["rho"])
    g.set_timeout(1e-7)
    with pytest.raises(LbmError) as ei:
        g.step(200)
    assert ei.value.status == LBM_ETIMEOUT
    g.set_timeout(600)
    g.check()
    assert g.t == 200


def test_set_fields_device_matches_host(cuda):
    torch = cuda
    c = cases.ragged(nx=64, ny=64)
    a = cases.gpu_sim(c)
    a.set_fields(c["rho"])
    a.step(10)
    b = cases.gpu_sim(c)
    b.set_fields_device(torch.from_numpy(c["rho"]).cuda())
    b.step(10)
    ra = a.fields()[0]
    rb = b.fields_device()[0].cpu().numpy()
    assert np.array_equal(ra, rb)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_timed_matches_step(cuda, precision):
    """lbm_step_timed (one step of direct launches with an event record around
    each pass) advances the state exactly like lbm_step, from either population
    buffer, and reports positive pass times (the FP64 path five, the mixed path
    four and a zero)."""
    c = cases.ragged(nx=64, ny=48)
    a = cases.gpu_sim(c, precision=precision)
    b = cases.gpu_sim(c, precision=precision)
    a.set_fields(c["rho"])
    b.set_fields(c["rho"])
    for _ in range(5):
        ms = a.step_timed()
        npass = 5 if precision == "fp64" else 4
        assert all(0 < m < 1e3 for m in ms[:npass])
        assert all(m >= 0 for m in ms)
    b.step(5)
    assert a.t == b.t == 5
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_mrt_steps_against_oracle(cuda, precision, tol):
    """MRT collision (Eq. 4, the paper's rates s_e 1.64, s_eps 1.54, s_q 1.9,
    s_v = 1/tau): the GPU's moment-space form against the oracle's literal
    f - M^-1 S M (f - f^eq) + F_i, after 301 steps of a ragged drop at T_r 0.7,
    k 0.3, tau 1 (with these rates the oracle itself blows up at T_r 0.6 for
    k >= 0.3, and at tau 0.8 for every k tried)."""
    from oracle import sim
    c = dict(cases.ragged(nx=48, ny=40, T_r=0.7), k=0.3, tau=1.0)
    g = cases.gpu_sim(c, precision=precision, collision="mrt")
    g.set_fields(c["rho"])
    g.step(301)
    o = cases.oracle_sim(c, mrt=sim.PAPER_MRT)
    o.set_fields(c["rho"])
    o.step(301)
    rho, vx, _, _ = g.fields()
    orho, ovx, _, _, _, _ = o.fields()
    assert rel_point(rho, orho) <= tol
    assert np.abs(vx - ovx).max() <= 1e2 * tol * np.abs(ovx).max()


def test_mrt_equal_rates_is_bgk_on_gpu(cuda):
    """With s_e = s_eps = s_q = 1/tau the MRT kernel computes the BGK collision
    (FP64, to rounding)."""
    c = cases.ragged(nx=40, ny=32)
    w = 1.0 / c["tau"]
    a = cases.gpu_sim(c)
    b = cases.gpu_sim(c, collision="mrt", mrt_rates=(w, w, w))
    a.set_fields(c["rho"])
    b.set_fields(c["rho"])
    a.step(100)
    b.step(100)
    assert rel_point(b.fields()[0], a.fields()[0]) <= 1e-12


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-4)])
def test_diagonal_slab_against_oracle(cuda, precision, tol):
    """A slab at 45 degrees to the grid (density a function of (x + y) mod n,
    periodic in both directions): both line directions cross the same
    interface.  200 steps against the oracle."""
    from oracle import OracleSim, thermo
    from paper_1906_09530_gb300 import Simulation
    n, tr, k = 64, 0.6, 0.5
    tc, _ = thermo.critical_point()
    rg, rl = thermo.maxwell(tr)
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    s = (x + y) % n
    rho = rg + (rl - rg) * 0.5 * (1 - np.tanh(2 * ((np.abs(s - n / 2) - n / 4) / np.sqrt(2)) / 8.0))
    g = Simulation(n, n, tr, 0.1, 1.0, k, fd_order=6, precision=precision)
    g.set_fields(rho)
    g.step(200)
    o = OracleSim(n, n, tr * tc, 0.1, 1.0, k, 6)
    o.set_fields(rho)
    o.step(200)
    assert rel_point(g.fields()[0], o.fields()[0]) <= tol
