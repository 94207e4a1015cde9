"""The other equations of state of Sec. 3.2 on the GPU: van der Waals (Eqs. 14-15),
Redlich-Kwong and its Soave form (Eqs. 16-17), Peng-Robinson (Eqs. 18-19),
against the FP64 oracle (oracle/eos.py, pinned by test_oracle_eos_variants.py).

Inputs: drops of radius 10 on a 48 x 40 grid at T_r = 0.7 with the paper's a, b
(omega = 0.344 for RKS and PR), kappa-hat = 0.005, k = 0.3, tau = 1, 6th order,
noise 1e-4.  These EOSs have liquid densities near 8, twenty times the CS
liquid, and kappa-hat is scaled down with them.  With kappa-hat = 0.1 or
k = 0.5 the oracle itself blows up (the short-wave sound speed k^2 p0' +
rho kappa theta'^2 passes c_s^2).  Tolerances are those of the CS parity tests.
"""
import numpy as np
import pytest

from oracle import OracleSim
from oracle import eos as E
from paper_1906_09530_gb300 import workloads as W

pytestmark = pytest.mark.gpu
KINDS = ["vdw", "rk", "rks", "pr"]
KAPPA, K, TR = 0.005, 0.3, 0.7


def _case(kind, nx=48, ny=40, T_r=TR):
    from paper_1906_09530_gb300 import make_eos
    omega = 0.344 if kind in ("rks", "pr") else 0.0
    o = E.Eos(kind, omega=omega)
    tc, _ = o.critical_point()
    rg, rl = o.maxwell(T_r)
    rho = W.with_noise(W.drop(nx, ny, rg, rl, 10.0, 4.0 / K), 7, 1e-4)
    return o, make_eos(kind, omega=omega), tc, rho


def _pair(kind, precision, nx=48, ny=40):
    from paper_1906_09530_gb300 import Simulation
    o, e, tc, rho = _case(kind, nx, ny)
    g = Simulation(nx, ny, TR, KAPPA, 1.0, K, fd_order=6, precision=precision, eos=e)
    g.set_fields(rho)
    s = OracleSim(nx, ny, TR * tc, KAPPA, 1.0, K, 6, eos=o)
    s.set_fields(rho)
    return g, s


def rel_point(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


@pytest.mark.parametrize("kind", KINDS)
def test_force_stage_t0_fp64(cuda, kind):
    g, s = _pair(kind, "fp64")
    rho, vx, vy, mu = g.fields()
    orho, ovx, ovy, omu, _, _ = s.fields()
    assert rel_point(rho, orho) <= 1e-14
    assert np.abs(mu - omu).max() <= 1e-12 * np.abs(omu).max()
    assert np.abs(vx - ovx).max() <= 1e-12 * np.abs(ovx).max()
    assert np.abs(vy - ovy).max() <= 1e-12 * np.abs(ovy).max()


@pytest.mark.parametrize("kind", KINDS)
def test_steps_fp64(cuda, kind):
    g, s = _pair(kind, "fp64")
    g.step(301)
    s.step(301)
    rho, vx, _, mu = g.fields()
    orho, ovx, _, omu, _, _ = s.fields()
    assert rel_point(rho, orho) <= 1e-10
    assert np.abs(vx - ovx).max() <= 1e-8 * np.abs(ovx).max()
    assert np.abs(mu - omu).max() <= 1e-8 * np.abs(omu).max()


@pytest.mark.parametrize("precision", ["mixed", "mixed_df"])
@pytest.mark.parametrize("kind", KINDS)
def test_mixed_close_to_oracle(cuda, kind, precision):
    g, s = _pair(kind, precision)
    rho, _, _, mu = g.fields()
    orho, _, _, omu, _, _ = s.fields()
    assert np.abs(mu - omu).max() <= 1e-5 * np.abs(omu).max()
    g.step(200)
    s.step(200)
    assert rel_point(g.fields()[0], s.fields()[0]) <= 1e-4


@pytest.mark.parametrize("kind", KINDS)
def test_batch_member_equals_lone_context(cuda, kind):
    """A batch with another EOS: every member equals a lone context bit for bit."""
    from paper_1906_09530_gb300 import Batch, Simulation
    o, e, tc, rho = _case(kind, 64, 48)
    o2, _, _, rho2 = _case(kind, 40, 56, T_r=0.8)
    spec = [dict(nx=64, ny=48, T_r=TR, kappa=KAPPA, k=K), dict(nx=40, ny=56, T_r=0.8,
                                                              kappa=KAPPA, k=K)]
    b = Batch(spec, eos=e)
    b.set_fields(0, rho)
    b.set_fields(1, rho2)
    b.step(9)
    for i, (d, r) in enumerate(zip(spec, (rho, rho2))):
        s = Simulation(d["nx"], d["ny"], d["T_r"], KAPPA, 1.0, K, fd_order=6,
                       precision="mixed", eos=e)
        s.set_fields(r)
        s.step(9)
        for x, y in zip(b.fields(i), s.fields()):
            assert np.array_equal(x, y)
        s.close()
    b.close()


@pytest.mark.parametrize("kind", KINDS)
def test_batch_coexistence(cuda, kind):
    """Sec. 5.1 / Fig. 4 for the other EOSs: flat interfaces (height 400, k = 0.1,
    kappa-hat = 0.005) at T_r = 0.6 and 0.8, run as one batch for 150 000 steps.
    Liquid within 1e-4 of Maxwell.  The gas sits above Maxwell by the scheme's
    offset, as for CS, and is bounded by 5%.  Measured at 200 000 steps: +0.4% to
    +1.8% at 0.6, +2e-4 to +2e-3 at 0.8 (VDW the least, PR the most), and the mixed
    path agrees with FP64 within 2e-4."""
    from paper_1906_09530_gb300 import Batch
    ny, k = 400, 0.1
    omega = 0.344 if kind in ("rks", "pr") else 0.0
    o = E.Eos(kind, omega=omega)
    _, e, _, _ = _case(kind)
    trs = (0.6, 0.8)
    b = Batch([dict(nx=8, ny=ny, T_r=t, k=k, kappa=KAPPA) for t in trs], eos=e)
    pairs = [o.maxwell(t) for t in trs]
    for i, (rg, rl) in enumerate(pairs):
        b.set_fields(i, W.flat(8, ny, rg, rl, ny / 2, 4.0 / k))
    b.step(150_000)
    for i, (rg, rl) in enumerate(pairs):
        r = b.fields(i)[0][:, 0]
        g = np.r_[r[: ny // 10], r[-ny // 10:]].mean()
        l = r[ny // 2 - ny // 20: ny // 2 + ny // 20].mean()
        assert abs(l / rl - 1) <= 1e-4
        assert -1e-3 <= g / rg - 1 <= 0.05
    b.close()


def _pole_field(ee, nx=48, ny=40):
    """A PR (or CS) drop with two nodes at and beyond the repulsive pole."""
    rg, rl = ee.maxwell(0.6)
    pole = 1.0 / (ee.b / 4.0 if ee.kind == "cs" else ee.b)
    rho = W.drop(nx, ny, rg, rl, 10.0, 4.0 / 0.2)
    rho[20, 24] = 1.02 * pole
    rho[21, 24] = pole
    return rho, pole


@pytest.mark.parametrize("kind,precision", [("pr", "fp64"), ("pr", "mixed"),
                                            ("cs", "fp64"), ("cs", "mixed")])
def test_upper_limit_takes_the_pole(cuda, kind, precision):
    """Sec. 5.6: while the limit acts, nodes at or beyond the pole get
    mu-hat = k^2 mu_max and the run goes on (FP64: as the oracle, step by
    step); with the limit off the same state is flagged unstable."""
    from paper_1906_09530_gb300 import LbmError, Simulation, make_eos
    ee = E.Eos(kind, omega=0.344 if kind == "pr" else 0.0)
    tc, _ = ee.critical_point()
    kappa, k, mu_max = (0.005, 0.2, 6.0) if kind == "pr" else (0.1, 0.5, 2.0)
    e = make_eos(kind, omega=0.344 if kind == "pr" else 0.0)
    rho, pole = _pole_field(ee)
    g = Simulation(48, 40, 0.6, kappa, 1.0, k, fd_order=6, precision=precision, eos=e,
                   mu_max=mu_max, mu_cap_steps=50)
    g.set_fields(rho)
    mu = g.fields()[3]
    cap = k * k * mu_max
    if precision == "fp64":
        assert mu[20, 24] == cap and mu[21, 24] == cap
    else:
        assert mu[20, 24] == pytest.approx(cap, rel=1e-7)
    g.step(5)
    if precision == "fp64":
        o = OracleSim(48, 40, 0.6 * tc, kappa, 1.0, k, 6, eos=None if kind == "cs" else ee,
                      mu_max=mu_max, mu_cap_steps=50)
        o.set_fields(rho)
        o.step(5)
        assert rel_point(g.fields()[0], o.fields()[0]) <= 1e-10
    g.close()
    with pytest.raises(LbmError):
        h = Simulation(48, 40, 0.6, kappa, 1.0, k, fd_order=6, precision=precision, eos=e)
        h.set_fields(rho)
        h.step(1)
