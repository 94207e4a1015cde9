"""Batched instances (lbm_batch_* of the C ABI): many independent periodic runs of
the mixed path advanced by one launch per pass.

Parity: within an instance a batch does the arithmetic of a lone context, block
for block, so every instance must equal a lone mixed Simulation on the same input
bit for bit (any difference would be a mapping error: a block given the wrong
instance, window or parameters).  The lone mixed path is itself pinned to the
oracle by test_gpu_parity.py; one batch member is also checked against the oracle
directly here.
"""
import math

import numpy as np
import pytest

from oracle import OracleSim, thermo
from paper_1906_09530_gb300 import workloads as W
from tests import cases

pytestmark = pytest.mark.gpu


def _instances():
    """Uneven sizes (ragged ones too), temperatures, k, tau, kappa; one with the
    upper limit on."""
    spec = [
        dict(nx=64, ny=64, T_r=0.7, k=0.5, tau=1.0, kappa=0.1),
        dict(nx=37, ny=29, T_r=0.6, k=0.5, tau=0.9, kappa=0.1),
        dict(nx=128, ny=96, T_r=0.5, k=0.35, tau=1.0, kappa=0.08),
        dict(nx=200, ny=168, T_r=0.45, k=0.5, tau=1.0, kappa=0.1),
        dict(nx=512, ny=512, T_r=0.55, k=0.5, tau=1.0, kappa=0.1),
        dict(nx=8, ny=400, T_r=0.8, k=0.1, tau=1.0, kappa=0.1),
        dict(nx=96, ny=96, T_r=0.45, k=0.5, tau=1.0, kappa=0.1, mu_cap_steps=5),
        # density ratios above 1e4: double-float density lines in "mixed" too
        dict(nx=160, ny=128, T_r=0.36, k=0.3, tau=1.0, kappa=0.1),
        dict(nx=8, ny=256, T_r=0.32, k=0.2, tau=1.0, kappa=0.1),
    ]
    tc = thermo.critical_point()[0]
    spec[6]["mu_max"] = float(thermo.mu0(0.5 * (1 + thermo.maxwell(0.45)[1]), 0.45 * tc))
    rhos = []
    for i, d in enumerate(spec):
        rg, rl = thermo.maxwell(d["T_r"])
        if d["nx"] == 8:
            r = W.flat(d["nx"], d["ny"], rg, rl, d["ny"] / 2, 4.0 / d["k"])
        else:
            r = W.drop(d["nx"], d["ny"], rg, rl, 0.25 * min(d["nx"], d["ny"]), 4.0 / d["k"])
        rhos.append(W.with_noise(r, 1000 + i, 1e-5))
    return spec, rhos


def _lone(d, rho, fd_order=6, precision="mixed"):
    from paper_1906_09530_gb300 import Simulation
    s = Simulation(d["nx"], d["ny"], d["T_r"], d["kappa"], d["tau"], d["k"], fd_order=fd_order,
                   precision=precision, mu_max=d.get("mu_max", math.inf),
                   mu_cap_steps=d.get("mu_cap_steps", 0))
    s.set_fields(rho)
    return s


@pytest.mark.parametrize("fd_order,steps,precision",
                         [(6, 7, "mixed"), (4, 10, "mixed"), (6, 5, "mixed_df")])
def test_batch_bitexact_vs_lone_contexts(cuda, fd_order, steps, precision):
    """Both density-line kinds (FP32 below ratio 1e4, double-float above, or
    double-float everywhere with "mixed_df") in one batch."""
    from paper_1906_09530_gb300 import Batch
    spec, rhos = _instances()
    b = Batch(spec, fd_order=fd_order, precision=precision)
    for i, r in enumerate(rhos):
        b.set_fields(i, r)
    b.step(steps)
    for i, (d, r) in enumerate(zip(spec, rhos)):
        s = _lone(d, r, fd_order, precision)
        s.step(steps)
        want = s.fields()
        got = b.fields(i)
        for name, x, y in zip(("rho", "vx", "vy", "mu"), got, want):
            assert np.array_equal(x, y), (i, name, np.abs(x - y).max())
        assert b.time(i) == steps
        s.close()
    b.close()


@pytest.mark.parametrize("nl", [8, 16])
def test_batch_lines_per_block_bitexact(cuda, nl):
    """The FP32 line launches with 8 or 16 lines a block give the lone contexts'
    results bit for bit (set before the first step and switched mid-run)."""
    from paper_1906_09530_gb300 import Batch
    spec, rhos = _instances()
    b = Batch(spec)
    b.set_lines_per_block(nl)
    assert b.lines_per_block() == nl
    for i, r in enumerate(rhos):
        b.set_fields(i, r)
    b.step(4)
    b.set_lines_per_block(24 - nl)
    b.step(3)
    for i, (d, r) in enumerate(zip(spec, rhos)):
        s = _lone(d, r)
        s.step(7)
        for x, y in zip(b.fields(i), s.fields()):
            assert np.array_equal(x, y), i
        s.close()
    b.close()


def test_batch_member_close_to_oracle(cuda):
    """A batch member against the FP64 oracle, at the lone mixed path's tolerance."""
    from paper_1906_09530_gb300 import Batch
    c = cases.config1()
    other = cases.ragged()
    b = Batch([dict(nx=c["nx"], ny=c["ny"], T_r=c["T_r"], k=c["k"], tau=c["tau"],
                    kappa=c["kappa"]),
               dict(nx=other["nx"], ny=other["ny"], T_r=other["T_r"], k=other["k"],
                    tau=other["tau"], kappa=other["kappa"])], fd_order=4)
    b.set_fields(0, c["rho"])
    b.set_fields(1, W.drop(other["nx"], other["ny"], *thermo.maxwell(other["T_r"]), 8.0, 4.0))
    b.step(200)
    o = cases.oracle_sim(c)
    o.set_fields(c["rho"])
    o.step(200)
    got, want = b.fields(0)[0], o.fields()[0]
    assert np.abs(got - want).max() / np.abs(want).max() <= 1e-4
    b.close()


def test_batch_autotune_keeps_state_and_results(cuda):
    """Autotuning times strip heights on the live state; the state is unchanged and
    the continued run still equals the lone contexts bit for bit."""
    from paper_1906_09530_gb300 import Batch
    spec, rhos = _instances()
    b = Batch(spec)
    for i, r in enumerate(rhos):
        b.set_fields(i, r)
    b.step(3)
    before = [b.fields(i) for i in range(len(spec))]
    b.autotune(reps=3)
    assert b.lines_per_block() in (8, 16)
    for i in range(len(spec)):
        assert b.tile_rows(i) in (4, 8, 16, 32)
        for x, y in zip(b.fields(i), before[i]):
            assert np.array_equal(x, y)
    b.step(4)
    for i, (d, r) in enumerate(zip(spec, rhos)):
        s = _lone(d, r)
        s.step(7)
        assert np.array_equal(b.fields(i)[0], s.fields()[0])
        s.close()
    b.close()


def test_batch_diag_and_time_levels(cuda):
    from paper_1906_09530_gb300 import Batch
    spec, rhos = _instances()
    b = Batch(spec)
    for i, r in enumerate(rhos):
        b.set_fields(i, r)
    b.step(5)
    mass, vmax, rmin, rmax = b.diag()
    for i, (d, r) in enumerate(zip(spec, rhos)):
        s = _lone(d, r)
        s.step(5)
        m, v, lo, hi = s.diag()
        assert mass[i] == pytest.approx(m, rel=1e-13)
        assert vmax[i] == pytest.approx(v, rel=1e-12)
        assert rmin[i] == lo and rmax[i] == hi
        s.close()
    # re-setting one instance restarts only its clock
    b.set_fields(2, rhos[2])
    assert b.time(2) == 0 and b.time(0) == 5
    b.step(2)
    assert b.time(2) == 2 and b.time(0) == 7
    b.close()


def test_batch_reports_the_failing_instance(cuda):
    """A bad density in instance 3 only: the step returns LBM_EUNSTABLE and names
    instance 3; after re-setting it the batch runs on."""
    from paper_1906_09530_gb300 import Batch, LbmError
    from paper_1906_09530_gb300._binding import LBM_EUNSTABLE
    spec, rhos = _instances()
    b = Batch(spec)
    for i, r in enumerate(rhos):
        if i == 3:
            bad = r.copy()
            bad[10, 20] = -1e-3
            with pytest.raises(LbmError):
                b.set_fields(i, bad)
        else:
            b.set_fields(i, r)
    inst, step = b.failed()
    assert inst == 3 and step == 0
    with pytest.raises(LbmError):  # instance 3 is unset: no step
        b.step(1)
    b.set_fields(3, rhos[3])
    b.step(4)
    bad = rhos[5].copy()
    with pytest.raises(LbmError) as ei:
        bad[100, 3] = float("nan")
        b.set_fields(5, bad)
        b.step(2)
    assert ei.value.status == LBM_EUNSTABLE
    assert b.failed()[0] == 5
    b.close()


def test_batch_rejects_bad_instances(cuda):
    from paper_1906_09530_gb300 import Batch, LbmError
    with pytest.raises(LbmError):
        Batch([dict(nx=64, ny=64, T_r=1.2)])
    with pytest.raises(LbmError):
        Batch([dict(nx=64, ny=4, T_r=0.7)])
    with pytest.raises(LbmError):
        Batch([dict(nx=64, ny=64, T_r=0.7, tau=0.5)])


def test_batch_step_timed_matches_step(cuda):
    from paper_1906_09530_gb300 import Batch
    spec, rhos = _instances()
    a, b = Batch(spec), Batch(spec)
    for i, r in enumerate(rhos):
        a.set_fields(i, r)
        b.set_fields(i, r)
    for _ in range(3):
        ms = a.step_timed()
        assert len(ms) == 4 and all(0 < m < 1e3 for m in ms)
    b.step(3)
    for i in range(len(spec)):
        assert np.array_equal(a.fields(i)[0], b.fields(i)[0])
    a.close()
    b.close()


def test_batch_mrt_bitexact_vs_lone(cuda):
    from paper_1906_09530_gb300 import Batch
    spec, rhos = _instances()
    spec, rhos = spec[:4], rhos[:4]
    b = Batch(spec, collision="mrt")
    for i, r in enumerate(rhos):
        b.set_fields(i, r)
    b.step(7)
    for i, (d, r) in enumerate(zip(spec, rhos)):
        from paper_1906_09530_gb300 import Simulation
        s = Simulation(d["nx"], d["ny"], d["T_r"], d["kappa"], d["tau"], d["k"], fd_order=6,
                       precision="mixed", mu_max=d.get("mu_max", math.inf),
                       mu_cap_steps=d.get("mu_cap_steps", 0), collision="mrt")
        s.set_fields(r)
        s.step(7)
        for x, y in zip(b.fields(i), s.fields()):
            assert np.array_equal(x, y)
        s.close()
    b.close()


def test_benchmark_batch_sampled_members_against_oracle(cuda):
    """The batch the benchmark times (256 instances, sides 64-512, T_r 0.3-0.9,
    drops and slabs, autotuned strip heights): after 3 steps, the smallest, the
    largest, the coldest (ratio above 1e10, double-float density lines) and a
    middle instance against the FP64 oracle, node by node."""
    from paper_1906_09530_gb300 import Batch
    specs = W.batch_instances(256)
    keys = ("nx", "ny", "T_r", "k", "kappa", "tau")
    b = Batch([{k: d[k] for k in keys} for d in specs])
    fields = [W.batch_field(d, *thermo.maxwell(d["T_r"])) for d in specs]
    for i, r in enumerate(fields):
        b.set_fields(i, r)
    b.autotune(3)
    b.step(3)
    sides = [d["nx"] for d in specs]
    picks = {sides.index(min(sides)), sides.index(max(sides)), 0, 128}
    tc = thermo.critical_point()[0]
    for i in sorted(picks):
        d = specs[i]
        o = OracleSim(d["nx"], d["ny"], d["T_r"] * tc, d["kappa"], d["tau"], d["k"], 6)
        o.set_fields(fields[i])
        o.step(3)
        got, want = b.fields(i)[0], o.fields()[0]
        assert np.max(np.abs(got - want) / want) <= 1e-5, (i, d["T_r"], d["nx"])
    b.close()
