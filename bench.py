#!/usr/bin/env python3
"""Benchmark of the chemical-potential multiphase LBM time step on GB300.

Workload (default): a 1024 x 1024 periodic static drop of radius 200 in its
Maxwell gas, Carnahan-Starling EOS (a=1, b=4, R=1) at T_r = 0.5, mesh
coefficient k = 0.5, 6th-order compact FD, tau = 1, kappa-hat = 0.1, tanh width
8, in the mixed precision path (FP32 populations, the density as an exact
double-float pair, double-float first derivatives of the density, FP32 for the
rest).  Synthetic, seeded inputs.

Also reported: `equilibrium`, the wall time from lbm_set_fields to
Maxwell-accurate equilibrium of a flat interface (see equilibrium_time);
`large_grid`, the same drop at 4096 x 4096 (working set far above L2), with
MRT, at 8192 x 8192, and in FP64; `batch`, 256 independent instances of uneven
sizes and temperatures advanced by one launch per pass (see batch_config); and
the two drop-splashing cases with walls (splash_config, splash_paper_config).

One "step" is one time step: the device passes of the chosen precision (mixed:
collide-stream, x|y compact FD of rho, pointwise chemical potential, x|y
compact FD of mu with the force; fp64: collide-stream and four single-axis line
passes).  Timing: W warm-up steps, then K steps, each bracketed by one pair of
CUDA events on the library's stream; between steps a 512 MB buffer is written
and another 512 MB read to flush the L2 (not timed).  value = nodes x K / sum
of step times.  The per-pass breakdown and the roofline come from a further
min(K, 200) flushed steps with events around every pass (lbm_step_timed).
e2e = the same metric through the public host API (lbm_set_fields from pinned
host memory, K steps, lbm_fields back to host), wall clock.  roofline: the
dominant pass against the measured copy bandwidth (frac) and the 7.9 TB/s
nominal (frac_nominal), with the whole step ("step") and the same figures at
4096^2 ("at_4096", working set far above L2).  cpu_baseline: the FP64 oracle on
all host cores (OpenMP), with its single-thread figure beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank runs its own replica (weak scaling, no collective
on the data path); rank 0 prints the JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = dict(nx=1024, ny=1024, T_r=0.5, k=0.5, kappa=0.1, tau=1.0, order=6, radius=200.0,
                width=8.0)
METRIC = "MLUPS (million lattice-node updates per second) of the full time step"
HBM_NOMINAL_GBS = 7900.0    # HBM3e nominal of one GB300, quoted beside the measured copy peak
FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (non-tensor) nominal: the FP64 path is bound by it
DF_RATIO = 1e4  # the mixed path's density lines are double-float from this Maxwell ratio


def pass_layout(precision, flags=0):
    """(names, algorithmic bytes per node) of the passes of one step (flags:
    lbm_path_flags).  Every field is read or written once per pass that needs
    it, in the precision the path stores it; x- and y-lines launched together
    are one pass.
      mixed, collide-stream: f 36 in + 36 out (FP32), F 8 in, rho hi/lo 8 out = 88
      x|y lines of rho: rho as hi/lo (8, double-float lines) or hi only (4) ->
        d_x, d_xx, d_y, d_yy 16
      mu-hat: rho_hi, d_xx, d_yy 12 -> mu 4 = 16
      x|y lines of mu-hat + force: mu 4, rho_hi 4, d_x, d_y 8 -> F 8 = 24
      fp64: collide 72 + 72 + F 16 + rho 8; x rho 8 -> 16; y rho, d_xx 16 -> 16;
      each force direction mu, rho, d rho 24 -> F 8."""
    if precision != "mixed":
        return (["collide_stream", "cfd_x_rho", "cfd_y_rho_mu", "cfd_x_force", "cfd_y_force"],
                [168, 24, 32, 32, 32])
    r = 8 if flags & 2 else 4
    return (["collide_stream", "cfd_rho_xy", "mu_pointwise", "cfd_mu_force_xy"],
            [88, r + 16, 16, 24])


def measured_traffic(precision):
    """DRAM bytes per node per launch from the committed ncu capture, if the
    kernel sources are unchanged since (else None)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic_mixed.json")
    if precision != "mixed" or not os.path.exists(p):
        return None
    d = json.load(open(p))
    h = hashlib.sha256(b"".join(open(os.path.join(ROOT, s), "rb").read()
                                for s in d["sources"])).hexdigest()[:16]
    return d["bytes_per_node"] if h == d["sources_sha256_16"] else None


def workload_name(w, precision):
    return (f"cs-drop-{w['nx']}x{w['ny']}-r{int(w['radius'])}-Tr{w['T_r']}-k{w['k']}"
            f"-cfd{w['order']}-{precision}")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.bus = bus_id
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            if self.bus and self.bus.lower()[-12:] not in parts[1].lower():
                continue
            rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def bus_id(dev):
    import torch
    p = torch.cuda.get_device_properties(dev)
    try:
        return f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}"
    except Exception:
        return None


def cpu_baseline(w, target_s=10.0):
    """The FP64 C oracle on a bounded sample of the same workload: as many
    full-grid time steps as fit in about target_s seconds, first on one thread,
    then with its loops over lines and nodes shared among all host cores
    (OpenMP).  `value` is the all-cores figure."""
    from oracle import OracleSim, sim as S, thermo
    from paper_1906_09530_gb300 import workloads as W
    Tc, _ = thermo.critical_point()
    rg, rl = thermo.maxwell(w["T_r"])
    rho = W.drop(w["nx"], w["ny"], rg, rl, w["radius"], w["width"])
    nproc = os.cpu_count() or 1

    def timed(threads):
        used = S.set_threads(threads)
        o = OracleSim(w["nx"], w["ny"], w["T_r"] * Tc, w["kappa"], w["tau"], w["k"],
                      w["order"])
        o.set_fields(rho)
        t0 = time.perf_counter()
        o.step(1)
        dt1 = time.perf_counter() - t0
        n = max(1, min(400, int(target_s / max(dt1, 1e-6)) - 1))
        t0 = time.perf_counter()
        o.step(n)
        dt = time.perf_counter() - t0
        return w["nx"] * w["ny"] * n / dt / 1e6, n, dt, used
    try:
        one, n1, dt1, _ = timed(1)
        allc, na, dta, used = timed(nproc)
    finally:
        S.set_threads(1)
    return {"value": allc, "unit": "MLUPS", "cores": used, "nproc": nproc, "kind": "oracle",
            "sample": f"{na} full {w['nx']}x{w['ny']} FP64 time steps of the same drop "
                      f"(after 1 untimed), plain C oracle, OpenMP over lines and nodes on "
                      f"{used} threads, {dta:.1f} s",
            "single_thread": {"value": one, "unit": "MLUPS", "cores": 1,
                              "sample": f"{n1} steps, 1 thread, {dt1:.1f} s"}}


EQ_WORKLOAD = dict(nx=8, ny=400, T_r=0.8, k=0.1, kappa=0.1, tau=1.0, order=6)


def equilibrium_time(precision, max_steps=600_000, nx=None, T_r=None):
    """Wall time from lbm_set_fields to Maxwell-accurate equilibrium of a flat
    interface (periodic, height 400, k = 0.1, T_r = 0.8 unless given; Sec. 5.1),
    quasi-1-D (8 wide) or nx wide.  Checked every 500 steps: done when the bulk
    gas (at the node farthest from both interfaces, where the oracle's fixed
    point reads it) and the bulk liquid (at the slab's centre) are both within
    1e-3 of the Maxwell pair and moved by < 1e-6 (relative) over the last 500
    steps.  (At k = 0.1 the method's own gas settles within 1e-3 of Maxwell only
    above T_r ~ 0.67: +7.2e-4 at 0.7, +3.5e-3 at 0.6, out of its reach at this
    k.)"""
    import numpy as np
    import paper_1906_09530_gb300 as P
    from paper_1906_09530_gb300 import workloads as W
    e = dict(EQ_WORKLOAD)
    if nx is not None:
        e["nx"] = nx
    if T_r is not None:
        e["T_r"] = T_r
    rg, rl = P.lbm_maxwell(e["T_r"])
    rho0 = W.flat(e["nx"], e["ny"], rg, rl, e["ny"] / 2, 4.0 / e["k"])
    sim = P.Simulation(e["nx"], e["ny"], e["T_r"], e["kappa"], e["tau"], e["k"],
                       fd_order=e["order"], precision=precision)
    ny = e["ny"]
    t0 = time.perf_counter()
    sim.set_fields(rho0)
    prev = None
    done = None
    while sim.t < max_steps:
        sim.step(500)
        r = sim.fields()[0][:, 0]
        g, l = r[0], r[ny // 2]
        cur = (g, l)
        if (prev is not None and abs(g / rg - 1) < 1e-3 and abs(l / rl - 1) < 1e-3
                and abs(g / prev[0] - 1) < 1e-6 and abs(l / prev[1] - 1) < 1e-6):
            done = time.perf_counter() - t0
            break
        prev = cur
    steps = sim.t
    sim.close()
    return {"workload": f"flat-interface-{e['nx']}x{ny}-Tr{e['T_r']}-k{e['k']}-{precision}",
            "wall_s": done, "steps": steps, "reached": done is not None,
            "gas_rel_err": float(cur[0] / rg - 1), "liquid_rel_err": float(cur[1] / rl - 1),
            "criterion": "both bulk densities (gas at the node farthest from both "
                         "interfaces, liquid at the slab centre) within 1e-3 of Maxwell and "
                         "steady to 1e-6 over 500 steps, checked every 500 steps"}


def large_grid(precision, steps, warmup, size=4096, collision="bgk", **over):
    """The bench drop scaled to size^2 (radius scaled with it): a working set far
    above the 129 MB L2, so no flush is needed.  Per-pass CUDA-event times and the
    step's algorithmic bytes against the measured copy bandwidth."""
    import numpy as np
    import paper_1906_09530_gb300 as P
    from paper_1906_09530_gb300 import workloads as W
    w = dict(WORKLOAD)
    s = size / w["nx"]
    w.update(nx=size, ny=size, radius=w["radius"] * s)
    w.update(over)
    rg, rl = P.lbm_maxwell(w["T_r"])
    sim = P.Simulation(w["nx"], w["ny"], w["T_r"], w["kappa"], w["tau"], w["k"],
                       fd_order=w["order"], precision=precision, collision=collision)
    sim.set_fields(W.drop(w["nx"], w["ny"], rg, rl, w["radius"], w["width"]))
    sim.step(warmup)
    names, pb = pass_layout(precision, sim.path_flags)
    ms = np.array([sim.step_timed() for _ in range(steps)])[:, :len(names)]
    sim.close()
    N = w["nx"] * w["ny"]
    step_ms = float(ms.sum(axis=1).mean())
    peak, peak_kind = load_peaks()
    gbs = sum(pb) * N / (step_ms / 1e3) / 1e9
    mean = ms.mean(axis=0)
    dom = int(np.argmax(mean))
    dom_gbs = pb[dom] * N / (float(mean[dom]) / 1e3) / 1e9
    return {"workload": workload_name(w, precision) + ("-mrt" if collision == "mrt" else ""),
            "collision": collision, "nodes": N, "steps": steps,
            "mlups": N / (step_ms / 1e3) / 1e6, "ms_per_step": step_ms,
            "passes_ms": {nm: round(float(mean[i]), 5) for i, nm in enumerate(names)},
            "passes_frac_hbm": {nm: round(pb[i] * N / (float(mean[i]) / 1e3) / 1e9 / peak, 4)
                                for i, nm in enumerate(names)},
            "dominant": {"kernel": names[dom], "alg_bytes_per_node": pb[dom],
                         "achieved_GB/s": dom_gbs, "frac": dom_gbs / peak},
            "step_roofline": {"alg_bytes_per_node": sum(pb), "achieved_GB/s": gbs,
                              "peak": peak, "frac": gbs / peak,
                              "peak_kind": f"{peak_kind} copy bandwidth"},
            "l2": "working set above L2 (no flush)"}


def fp64_path_summary(lg):
    """The FP64 path at 4096^2 against the FP64 pipe: its FP64 operations per
    node (FMA counted as two) from the committed ncu count, if the kernel sources
    are unchanged since, times the node rate, over the GB300's FP64 nominal."""
    out = {"workload": lg["workload"], "mlups": lg["mlups"],
           "frac_hbm": lg["step_roofline"]["frac"], "bound": "fp64 pipe"}
    import hashlib
    p = os.path.join(ROOT, "profiles", "fp64_ops.json")
    if os.path.exists(p):
        d = json.load(open(p))
        h = hashlib.sha256(b"".join(open(os.path.join(ROOT, f), "rb").read()
                                    for f in d["sources"])).hexdigest()[:16]
        if h == d["sources_sha256_16"]:
            fl = d["fp64_flops_per_node"]
            tf = fl * lg["mlups"] * 1e6 / 1e12
            out.update({"fp64_flops_per_node": fl, "achieved_tflops": tf,
                        "peak_tflops": FP64_NOMINAL_TFLOPS, "frac": tf / FP64_NOMINAL_TFLOPS,
                        "peak_kind": "nominal"})
    return out


def batch_config(steps, warmup, n=256):
    """The batched path on many independent instances (uneven sides 64-512, T_r
    log-spaced 0.3-0.9, drops and flat interfaces; workloads.batch_instances):
    one launch per pass for all of them, strip heights and the FP32 line
    launches' lines per block autotuned.  Compared with
    the same instances stepped one after another as lone contexts (each with its
    own two-step CUDA graph)."""
    import numpy as np
    import torch
    import paper_1906_09530_gb300 as P
    from paper_1906_09530_gb300 import workloads as W
    specs = W.batch_instances(n)
    keys = ("nx", "ny", "T_r", "k", "kappa", "tau")
    b = P.Batch([{k: d[k] for k in keys} for d in specs])
    fields = []
    for i, d in enumerate(specs):
        fields.append(W.batch_field(d, *P.lbm_maxwell(d["T_r"])))
        b.set_fields(i, fields[-1])
    b.autotune(3)
    chosen_nl = b.lines_per_block()
    b.step(warmup)
    # the line launches' lines per block, each way (the autotuner keeps the faster)
    names = pass_layout("mixed")[0]
    nl_passes = {}
    for nl in (8, 16):
        b.set_lines_per_block(nl)
        b.step(2)
        m2 = np.array([b.step_timed() for _ in range(min(steps, 20))])
        nl_passes[nl] = {nm: round(float(m2[:, i].mean()), 5) for i, nm in enumerate(names)}
    b.set_lines_per_block(chosen_nl)
    ms = np.array([b.step_timed() for _ in range(steps)])
    N = sum(d["nx"] * d["ny"] for d in specs)
    step_ms = float(ms.sum(axis=1).mean())
    # graph replay of the whole batch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kb = max(2, steps // 2 * 2)
    torch.cuda.synchronize()
    e0.record()
    b.step(kb)
    e1.record()
    torch.cuda.synchronize()
    graph_ms = e0.elapsed_time(e1) / kb
    b.close()
    # the same instances as lone contexts, one after another
    sims = []
    for d, r in zip(specs, fields):
        s = P.Simulation(d["nx"], d["ny"], d["T_r"], d["kappa"], d["tau"], d["k"], fd_order=6,
                         precision="mixed")
        s.set_fields(r)
        s.step(2)
        sims.append(s)
    torch.cuda.synchronize()
    e0.record()
    for s in sims:
        s.step_async(2)
    e1.record()
    torch.cuda.synchronize()
    lone_ms = e0.elapsed_time(e1) / 2
    for s in sims:
        s.check()
        s.close()
    # batches run the merged passes; double-float density lines from DF_RATIO
    alg = 0
    for d in specs:
        rg, rl = P.lbm_maxwell(d["T_r"])
        alg += d["nx"] * d["ny"] * sum(pass_layout("mixed", 2 if rl >= DF_RATIO * rg else 0)[1])
    pb = alg / N
    peak, peak_kind = load_peaks()
    return {"workload": f"batch-{n}-instances-sides64-512-Tr0.3-0.9-mixed", "instances": n,
            "nodes": N, "steps": steps,
            "mlups": N / (step_ms / 1e3) / 1e6,
            "graph_mlups": N / (graph_ms / 1e3) / 1e6,
            "lone_sequential_mlups": N / (lone_ms / 1e3) / 1e6,
            "passes_ms": {nm: round(float(ms[:, i].mean()), 5)
                          for i, nm in enumerate(pass_layout("mixed")[0])},
            "step_roofline": {"alg_bytes_per_node": pb,
                              "frac": pb * N / (step_ms / 1e3) / 1e9 / peak,
                              "peak": peak, "peak_kind": f"{peak_kind} copy bandwidth"},
            "launches_per_step": 4,
            "lines_per_block": chosen_nl,
            "passes_ms_by_lines_per_block": nl_passes,
            "l2": "working set above L2 (no flush)"}


SPLASH = dict(nx=2048, ny=1024, T_r=0.55, k=0.5, kappa=0.1, tau=1.0, order=6, film=100,
              radius=100.0, height=200.0, width=8.0, u_drop=-0.1, u_shift=0.05)


def spreading_radius(rho, y, xc, mid):
    """Spreading radius of an impact at column xc, read on row y: from xc go
    each way across any gas (the crater) to the outer edge of the first liquid
    run (the rim); half the distance between the two edges, 0 if the row holds
    no liquid within half the width."""
    import numpy as np
    row = np.asarray(rho[y]) > mid
    n = row.size

    def edge(step):
        d = 0
        while d < n // 2 and not row[(xc + step * d) % n]:
            d += 1
        if d >= n // 2:
            return None
        while d < n // 2 and row[(xc + step * d) % n]:
            d += 1
        return d - 1

    r, l = edge(1), edge(-1)
    return 0.0 if r is None or l is None else (r + l + 1) / 2.0


def phase_mismatch(a, b, mid):
    """Nodes on different sides of the midpoint density in a and b, and the
    interface links of a (the mean outline displacement is their ratio)."""
    import numpy as np
    pa, pb = a > mid, b > mid
    links = int((np.diff(pa.astype(np.int8), axis=1) != 0).sum() +
                (np.diff(pa.astype(np.int8), axis=0) != 0).sum())
    return int((pa != pb).sum()), links


def spread_fit(tstar, r, D, lo=0.5, hi=3.0):
    """(C, exponent) of r/D = C (t*)^e over lo <= t* <= hi: C by least squares
    with e = 1/2, e from the log-log slope.  A sample below 3/4 of the median
    of its five neighbours is dropped (the probe row met a bubble or a drop
    instead of the rim)."""
    import numpy as np
    tstar, r = np.asarray(tstar, dtype=np.float64), np.asarray(r, dtype=np.float64)
    med = np.array([np.median(r[max(0, i - 2):i + 3]) for i in range(r.size)])
    sel = (tstar >= lo) & (tstar <= hi) & (r > 0) & (r >= 0.75 * med)
    if sel.sum() < 3:
        return None, None
    sq = np.sqrt(tstar[sel])
    C = float((r[sel] / D) @ sq / (sq @ sq))
    e = float(np.polyfit(np.log(tstar[sel]), np.log(r[sel] / D), 1)[0])
    return C, e


def splash_config(precision="mixed", steps=10_000, every=100):
    """Drop splashing (Sec. 5.5): a drop of diameter 200 falling at 0.1 onto a
    film of thickness 100 on the bottom wall of a 2048 x 1024 channel (periodic
    in x, walls in y), CS T_r 0.55, k 0.5, tau 1 (Re = U D / nu = 120); once in
    a static frame and once in a frame moving at 0.05 (fluid and walls), run
    side by side.  Reports throughput (CUDA events around the stepping only),
    mass drift, the spreading radius r(t) on the row four nodes above the film
    against r/D = C sqrt(U t / D) after impact (spread_fit, t* = U t / D from 0.5
    to 3, t from the nominal contact, (height - radius) / U), and the outline
    mismatch between the two frames over time."""
    import numpy as np
    import torch
    import paper_1906_09530_gb300 as P
    from paper_1906_09530_gb300 import workloads as W
    c = SPLASH
    nx, ny = c["nx"], c["ny"]
    rg, rl = P.lbm_maxwell(c["T_r"])
    mid = 0.5 * (rg + rl)
    D, U = 2 * c["radius"], -c["u_drop"]
    t_c = (c["height"] - c["radius"]) / U
    yprobe = c["film"] + 4
    frames = (("static", 0.0), ("moving_frame", c["u_shift"]))
    sims, m0 = {}, {}
    for name, us in frames:
        sims[name] = P.Simulation(nx, ny, c["T_r"], c["kappa"], c["tau"], c["k"],
                                  fd_order=c["order"], precision=precision, walls_y=True,
                                  wall_ux=(us, us))
        sims[name].set_fields(*W.splash(nx, ny, rg, rl, c["film"], c["radius"], c["height"],
                                        c["width"], c["u_drop"], us))
        m0[name] = sims[name].diag()[0]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ms = {n: 0.0 for n, _ in frames}
    rs = {n: [] for n, _ in frames}
    ts, gal = [], {}
    for k in range(steps // every):
        rho = {}
        for name, us in frames:
            sim = sims[name]
            torch.cuda.synchronize()
            ev[0].record()
            sim.step(every)
            ev[1].record()
            torch.cuda.synchronize()
            ms[name] += ev[0].elapsed_time(ev[1])
            rho[name] = sim.fields()[0]
            xc = int(round(nx / 2 + us * sim.t)) % nx
            rs[name].append(spreading_radius(rho[name], yprobe, xc, mid))
        t = sims["static"].t
        ts.append(t)
        tstar = U * (t - t_c) / D
        if (k + 1) % 10 == 0:
            shifted = np.roll(rho["moving_frame"], -int(round(c["u_shift"] * t)), axis=1)
            bad, links = phase_mismatch(rho["static"], shifted, mid)
            gal[f"{tstar:.2f}"] = {"mismatch_nodes": bad, "interface_links": links}
    ts = np.array(ts, dtype=np.float64)
    tstar = U * (ts - t_c) / D
    res = {}
    for name, _ in frames:
        sim = sims[name]
        m1, vmax = sim.diag()[:2]
        sim.close()
        r = np.array(rs[name])
        C, expo = spread_fit(tstar, r, D)
        res[name] = {"mlups": nx * ny * steps / (ms[name] / 1e3) / 1e6,
                     "ms_per_step": ms[name] / steps,
                     "mass_rel_drift": abs(m1 - m0[name]) / m0[name], "max_v_end": vmax,
                     "spread_C": C, "spread_exponent": expo,
                     "r_over_D": {f"{a:.2f}": round(float(b / D), 4)
                                  for a, b in zip(tstar[4::5], r[4::5]) if a > 0}}
    return {"workload": f"splash-{nx}x{ny}-D{int(D)}-U{U}-film{c['film']}-Tr{c['T_r']}"
                        f"-k{c['k']}-{precision}",
            "steps": steps, "density_ratio": rl / rg, "reynolds": U * D / ((c["tau"] - 0.5) / 3),
            **res,
            "galilean": {"frame_speed": c["u_shift"], "by_tstar": gal},
            "timing": "CUDA events around lbm_step chunks of 100 steps; fields read "
                      "between chunks (not timed)"}


SPLASH_PAPER = dict(nx=1000, ny=300, T_r=0.6, k=0.1, kappa=0.005, order=6, film=30,
                    radius=50.0, gap=25.0, u_drop=-0.1, omega=0.344, mu_max=6.0,
                    mu_cap_steps=1000, frame=0.03)


def splash_paper_config(t_end=7.6, every=100):
    """The paper's own drop-splashing case (Sec. 5.5, Figs. 10-12): PR water
    (omega 0.344) at T_r 0.6, 1000 x 300 (periodic x, walls in y), D = 100,
    U = 0.1, film 30, k = 0.1, kappa-hat 0.005, mixed path; Re = U D / nu = 40
    (tau 1.25) and 150 (tau 0.7), the upper limit mu_max = 6 for the first 1000
    steps (Sec. 5.6), and Re 150 again in a frame moving at 0.03.  The drop
    starts 25 nodes above the film.  Reports the spreading constant C and
    exponent (spread_fit, t* 0.5-3), r/D at t* = 1..7, the outline mismatch of
    the moving frame at the paper's snapshot times, and throughput."""
    import numpy as np
    import torch
    import paper_1906_09530_gb300 as P
    from paper_1906_09530_gb300 import workloads as W
    c = SPLASH_PAPER
    nx, ny = c["nx"], c["ny"]
    eos = P.make_eos("pr", omega=c["omega"])
    rg, rl = P.lbm_maxwell(c["T_r"], eos)
    mid = 0.5 * (rg + rl)
    D, U = 2 * c["radius"], -c["u_drop"]
    t_c = c["gap"] / U
    steps = int(round((t_c + t_end * D / U) / every)) * every
    snap_t = [int(t_c + ts * D / U) // every * every for ts in (0.5, 2.0, 4.5, 7.6)]
    res, snaps = {}, {}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for name, tau, us in (("re40", 1.25, 0.0), ("re150", 0.7, 0.0),
                          ("re150_frame", 0.7, c["frame"])):
        sim = P.Simulation(nx, ny, c["T_r"], c["kappa"], tau, c["k"], fd_order=c["order"],
                           precision="mixed", eos=eos, mu_max=c["mu_max"],
                           mu_cap_steps=c["mu_cap_steps"], walls_y=True, wall_ux=(us, us))
        sim.set_fields(*W.splash(nx, ny, rg, rl, c["film"], c["radius"],
                                 c["radius"] + c["gap"], 2.0 / c["k"], c["u_drop"], us))
        m0 = sim.diag()[0]
        ms, ts, rs = 0.0, [], []
        snaps[name] = {}
        while sim.t < steps:
            torch.cuda.synchronize()
            ev[0].record()
            sim.step(every)
            ev[1].record()
            torch.cuda.synchronize()
            ms += ev[0].elapsed_time(ev[1])
            rho = sim.fields()[0]
            xc = int(round(nx / 2 + us * sim.t)) % nx
            ts.append(sim.t)
            rs.append(spreading_radius(rho, c["film"] + 5, xc, mid))
            if sim.t in snap_t:
                snaps[name][sim.t] = np.roll(rho, -int(round(us * sim.t)), axis=1) > mid
        m1 = sim.diag()[0]
        sim.close()
        tstar = U * (np.array(ts, dtype=np.float64) - t_c) / D
        r = np.array(rs)
        C, e = spread_fit(tstar, r, D)
        res[name] = {"reynolds": U * D / ((tau - 0.5) / 3), "tau": tau, "spread_C": C,
                     "spread_exponent": e, "mass_rel_drift": abs(m1 - m0) / m0,
                     "mlups": nx * ny * steps / (ms / 1e3) / 1e6,
                     "r_over_D": {f"{a:.1f}": round(float(b / D), 3) for a, b in zip(tstar, r)
                                  if a > 0.9 and abs(a - round(a)) < 0.051}}
    gal = {}
    for t in snap_t:
        a, b = snaps["re150"].get(t), snaps["re150_frame"].get(t)
        if a is not None and b is not None:
            links = int((np.diff(a.astype(np.int8), axis=1) != 0).sum() +
                        (np.diff(a.astype(np.int8), axis=0) != 0).sum())
            gal[f"{U * (t - t_c) / D:.2f}"] = {"mismatch_nodes": int((a != b).sum()),
                                               "interface_links": links}
    return {"workload": f"splash-paper-{nx}x{ny}-D{int(D)}-U{U}-film{c['film']}-PR-Tr{c['T_r']}"
                        f"-k{c['k']}-cap{c['mu_max']}x{c['mu_cap_steps']}-mixed",
            "density_ratio": rl / rg, "steps": steps, **res,
            "galilean_frame_0.03_re150": gal,
            "paper_reference": "2-D spreading constant C about 1.3 (Sec. 5.5)"}


def surrogate_demo():
    """The learned warm start: a surrogate trained on 256 equilibrium slabs
    (T_r 0.33-0.5, kappa-hat 0.1, k 0.2) by the library's MLP kernels, then
    steps and wall time to equilibrium (both bulks within the tolerance of a
    1.5M-step run) from the tanh start and from the warm start, on a tall slab
    (8 x 1536) where the gas offset relaxes by slow diffusion; and at T_r 0.35
    the 4096^2 drop of radius 1000 from both starts (warm_drop_case).  Also
    the training step's tensor throughput (BF16 products, FP32 accumulation)."""
    import numpy as np
    import torch
    from paper_1906_09530_gb300 import Simulation, lbm_maxwell, surrogate as SG
    from paper_1906_09530_gb300 import workloads as W
    ranges = {"T_r": (0.33, 0.5), "kappa": (0.1, 0.1), "k": (0.2, 0.2)}
    n = 256
    T = np.linspace(*ranges["T_r"], n)
    K, k = np.full(n, 0.1), np.full(n, 0.2)
    t0 = time.perf_counter()
    G, L, P = SG.equilibrium_profiles(T, K, k, steps=200_000)
    data_s = time.perf_counter() - t0
    s = SG.Surrogate(seed=3, ranges=ranges)
    t0 = time.perf_counter()
    loss = s.fit(T, K, k, G, L, P, epochs=3000, lr=2e-3, batch=128)
    fit_s = time.perf_counter() - t0
    # training-step throughput at batch 256 (algorithmic flops: forward
    # 2 (4*256 + 3*256^2) per sample, backward twice that less the input layer's
    # input gradient)
    # timed on a network of its own, so the trained one is left as it is
    from paper_1906_09530_gb300 import Mlp
    tnet = Mlp(256)
    tnet.set_params(SG.glorot_params(0))
    x = torch.rand((256, 4), device="cuda") * 2 - 1
    y = torch.rand((256, 256), device="cuda")
    for _ in range(10):
        tnet.train_step(x, y, 1e-3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(200):
        tnet.train_step(x, y, 1e-3)
    e1.record()
    torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / 200
    tnet.close()
    fwd = 2 * (4 * 256 + 3 * 256 * 256)
    flops = 256 * (fwd + 2 * fwd - 2 * 4 * 256)
    peak, _ = load_bf16_peak()
    tflops = flops / (step_ms / 1e3) / 1e12
    ny = 1536

    def bulk(sim):
        r = sim.fields()[0][:, 0]
        return (np.r_[r[: ny // 10], r[-ny // 10:]].mean(),
                r[ny // 2 - ny // 10: ny // 2 + ny // 10].mean())
    cases = []
    for t_r in (0.35, 0.42):
        rg, rl = lbm_maxwell(t_r)
        ref = Simulation(8, ny, t_r, 0.1, 1.0, 0.2, fd_order=6, precision="mixed")
        ref.set_fields(W.flat(8, ny, rg, rl, ny / 2, 20.0))
        ref.step(1_500_000)
        eq = bulk(ref)
        ref.close()
        g, l, w = s.predict([t_r], [0.1], [0.2])
        row = {"T_r": t_r, "gas_offset_vs_maxwell": eq[0] / rg - 1,
               "predicted_gas_rel_err": g[0] / eq[0] - 1, "predicted_liq_rel_err": l[0] / eq[1] - 1}
        for name, field in (("tanh", W.flat(8, ny, rg, rl, ny / 2, 20.0)),
                            ("warm", SG.flat_field(8, ny, g[0], l[0], w[0]))):
            for tol in (1e-2, 1e-3):
                sim = Simulation(8, ny, t_r, 0.1, 1.0, 0.2, fd_order=6, precision="mixed")
                sim.set_fields(field)
                c0 = time.perf_counter()
                n_steps = SG.steps_to_equilibrium(sim, bulk, eq, tol, every=2000,
                                                  max_steps=1_000_000)
                row[f"{name}_steps_to_{tol:g}"] = n_steps
                row[f"{name}_wall_s_to_{tol:g}"] = time.perf_counter() - c0
                sim.close()
        cases.append(row)
        if t_r == 0.35:
            cases.append(warm_drop_case(s, eq, t_r))
    cases.append(coexistence_curve_case(s))
    s.close()
    return {"workload": "slab-8x1536-k0.2-kappa0.1, surrogate trained on 256 slabs T_r 0.33-0.5",
            "training_data_s": data_s, "fit_s": fit_s, "fit_loss": loss,
            "train_step_ms_batch256": step_ms,
            "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                         "frac": tflops / peak,
                         "note": "256-wide products: latency-bound, microseconds per step"},
            "cases": cases}


def collide_forms(sizes=(1024, 2048, 4096), reps=50):
    """The mixed collide-stream pass alone in each of its forms (sliding window,
    row ring with 8, 16 or 32 rows a block, the default choice) on the bench drop
    at each size: CUDA-event times of the pass (lbm_step_timed), the L2 flushed
    before every step as in the main timing.  88 algorithmic bytes a node (nine FP32 populations and
    the force read and written back, the density pair written)."""
    import numpy as np
    import torch
    import paper_1906_09530_gb300 as P
    from paper_1906_09530_gb300 import workloads as W
    peak, how = load_peaks()
    # the main timing's flush: dirty lines written, then evicted by a clean read,
    # so the timed pass pays no write-back of the flush itself
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    clean = torch.zeros(128 << 20, dtype=torch.float32, device="cuda")
    out = {"peak_GB/s": peak, "peak_kind": how, "alg_bytes_per_node": 88, "rows": []}
    for size in sizes:
        w = dict(WORKLOAD)
        sc = size / w["nx"]
        w.update(nx=size, ny=size, radius=w["radius"] * sc)
        rg, rl = P.lbm_maxwell(w["T_r"])
        sim = P.Simulation(w["nx"], w["ny"], w["T_r"], w["kappa"], w["tau"], w["k"],
                           fd_order=w["order"], precision="mixed")
        sim.set_fields(W.drop(w["nx"], w["ny"], rg, rl, w["radius"], w["width"]))
        sim.step(4)
        N = size * size
        row = {"size": size}
        for name, form in (("sliding_window", -1), ("ring_rows8", 8), ("ring_rows16", 16),
                           ("ring_rows32", 32), ("default", 0)):
            sim.set_collide_form(form)
            ms = []
            for _ in range(reps + 3):
                flush.zero_()
                clean.amax()
                ms.append(sim.step_timed()[0])
            us = float(np.mean(ms[3:])) * 1e3
            row[name + "_us"] = round(us, 2)
            row[name + "_frac"] = round(88 * N / (us / 1e6) / 1e9 / peak, 4)
        row["default_is_ring"] = bool(sim.path_flags & 4)
        sim.close()
        out["rows"].append(row)
    return out


def launch_overlap(steps=300, graph_steps=2000):
    """How a step's passes are launched, on the bench drop at 1024^2, in one
    process: lone steps (lbm_step_async of one step) launched directly or from a
    one-step graph, each with programmatic dependent launch off and on, each
    step bracketed by an event pair with the L2 flushed between steps as in the
    main timing; and back-to-back graph replays, without flushing, with it off
    and on."""
    import numpy as np
    import torch
    import paper_1906_09530_gb300 as P
    from paper_1906_09530_gb300 import workloads as W
    w = dict(WORKLOAD)
    rg, rl = P.lbm_maxwell(w["T_r"])
    sim = P.Simulation(w["nx"], w["ny"], w["T_r"], w["kappa"], w["tau"], w["k"],
                       fd_order=w["order"], precision="mixed")
    sim.set_fields(W.drop(w["nx"], w["ny"], rg, rl, w["radius"], w["width"]))
    N = w["nx"] * w["ny"]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    clean = torch.zeros(128 << 20, dtype=torch.float32, device="cuda")
    out = {"workload": workload_name(w, "mixed"), "lone_step_us": {}, "graph_mlups": {}}

    def lone(mode):
        sim.set_launch_mode(*mode)
        sim.step(10)
        ea = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        eb = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        for i in range(steps):
            flush.zero_()
            clean.amax()
            ea[i].record()
            sim.step_async(1)
            eb[i].record()
        sim.check()
        return float(np.mean([a.elapsed_time(b) for a, b in zip(ea, eb)])) * 1e3

    for rep in range(2):
        for name, mode in (("direct", (0, 0, 0)), ("direct_pdl", (0, 1, 0)),
                           ("graph", (1, 0, 0)), ("graph_pdl", (1, 0, 1))):
            out["lone_step_us"].setdefault(name, []).append(round(lone(mode), 2))
        for name, mode in (("off", (0, 0, 0)), ("pdl", (0, 0, 1))):
            sim.set_launch_mode(*mode)
            sim.step(16)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            sim.step_async(graph_steps)
            e1.record()
            sim.check()
            out["graph_mlups"].setdefault(name, []).append(
                round(N * graph_steps / (e0.elapsed_time(e1) / 1e3) / 1e6, 1))
    sim.close()
    return out


def mlp_products(batches=(256, 4096, 32768), reps=50):
    """The surrogate network's kernels alone: forward pass and Adam training
    step at several batch sizes, with the forward and input-gradient products
    on tcgen05 (the default) and on the mma.sync comparison kernel.
    Algorithmic flops per sample: forward 2 (4*256 + 3*256^2); training step
    three times that less the input layer's input gradient (2*4*256)."""
    import torch
    from paper_1906_09530_gb300 import Mlp, surrogate as SG
    peak, how = load_bf16_peak()
    fwd = 2 * (4 * 256 + 3 * 256 * 256)
    train = 3 * fwd - 2 * 4 * 256
    out = {"peak_tflops": peak, "peak_kind": how, "rows": []}
    for B in batches:
        net = Mlp(B)
        net.set_params(SG.glorot_params(0))
        g = torch.Generator(device="cuda").manual_seed(B)
        x = torch.rand((B, 4), device="cuda", generator=g) * 2 - 1
        t = torch.rand((B, 256), device="cuda", generator=g)
        row = {"batch": B}
        for tc in (True, False):
            net.tcgen05 = tc
            name = "tcgen05" if tc else "mma_sync"
            for what, call, flops in (("forward", lambda: net.forward(x), fwd),
                                      ("train_step", lambda: net.train_step(x, t, 1e-4), train)):
                for _ in range(5):
                    call()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                for _ in range(reps):
                    call()
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                tf = B * flops / (ms / 1e3) / 1e12
                row[f"{what}_{name}_us"] = ms * 1e3
                row[f"{what}_{name}_tflops"] = tf
                row[f"{what}_{name}_frac"] = tf / peak
            assert net.tcgen05 == tc  # no fall back happened
        net.close()
        out["rows"].append(row)
    return out


def windowed_equilibrium(step, sample, targets, tol, every, window, max_steps):
    """Steps until the means of the last `window` samples of every item are
    within tol (relative) of its target pair.  sample() returns one (gas,
    liquid) pair per item; a sample is taken, then `every` steps are run, until
    max_steps.  Returns (steps, means [item][2]) or (None, the last means)."""
    import numpy as np
    hist, t = [], 0
    while t < max_steps:
        hist.append(sample())
        if len(hist) >= window:
            m = np.mean(np.array(hist[-window:]), axis=0)
            if all(abs(m[j][0] / g - 1) <= tol and abs(m[j][1] / l - 1) <= tol
                   for j, (g, l) in enumerate(targets)):
                return t, m
        step(every)
        t += every
    return None, np.mean(np.array(hist[-window:]), axis=0)


def coexistence_curve_case(s, n=16, ny=1536, tol=1e-3, every=500, window=16,
                           max_steps=300_000):
    """A coexistence curve of n temperatures (T_r 0.35-0.48, kappa-hat 0.1, k 0.2,
    flat slabs 8 x ny), two ways, each until both bulk densities of every slab,
    averaged over the last `window` samples taken every `every` steps, are
    within tol of the method's own equilibrium (a batched 300 000-step run of
    8 x 384 slabs at the same parameters; the gas never reaches Maxwell at these
    temperatures).  The average filters the acoustic waves of the tall liquid
    layer, which viscosity damps only over about 3e5 steps and which a single
    sample would alias.
      plain: one lone context per temperature from the tanh start, one after
             another;
      batched: one batch of all n from the tanh starts (batching alone);
      batched + warm: one batch of all n from the surrogate's warm starts.
    Wall times are the host clock around the stepping and the sampling."""
    import numpy as np
    from paper_1906_09530_gb300 import Batch, Simulation, lbm_maxwell, surrogate as SG
    from paper_1906_09530_gb300 import workloads as W
    T = np.linspace(0.35, 0.48, n)
    K, k = np.full(n, 0.1), np.full(n, 0.2)
    G, L, _ = SG.equilibrium_profiles(T, K, k, steps=300_000)

    def bulk(r):
        return (np.r_[r[: ny // 10], r[-ny // 10:]].mean(),
                r[ny // 2 - ny // 10: ny // 2 + ny // 10].mean())

    def run(step, sample, idx):
        """Steps until the windowed means of every listed slab are within tol."""
        return windowed_equilibrium(step, lambda: [sample(i) for i in idx],
                                    [(G[i], L[i]) for i in idx], tol, every, window, max_steps)
    t0 = time.perf_counter()
    plain_steps = []
    for i, t in enumerate(T):
        rg, rl = lbm_maxwell(float(t))
        sim = Simulation(8, ny, float(t), 0.1, 1.0, 0.2, fd_order=6, precision="mixed")
        sim.set_fields(W.flat(8, ny, rg, rl, ny / 2, 20.0))
        st, _ = run(sim.step, lambda _i: bulk(sim.fields()[0][:, 0]), [i])
        plain_steps.append(st)
        sim.close()
    plain_s = time.perf_counter() - t0
    specs = [dict(nx=8, ny=ny, T_r=float(t), k=0.2, kappa=0.1, tau=1.0) for t in T]
    # batched, tanh starts (what batching alone gains)
    t0 = time.perf_counter()
    b = Batch(specs)
    for i, t in enumerate(T):
        b.set_fields(i, W.flat(8, ny, *lbm_maxwell(float(t)), ny / 2, 20.0))
    tanh_steps, _ = run(b.step, lambda i: bulk(b.fields(i)[0][:, 0]), list(range(n)))
    batch_tanh_s = time.perf_counter() - t0
    b.close()
    # batched, warm starts
    t0 = time.perf_counter()
    g, l, w = s.predict(T, K, k)
    b = Batch(specs)
    for i in range(n):
        b.set_fields(i, SG.flat_field(8, ny, g[i], l[i], w[i]))
    steps, m = run(b.step, lambda i: bulk(b.fields(i)[0][:, 0]), list(range(n)))
    batch_s = time.perf_counter() - t0
    b.close()
    worst = float(max(max(abs(m[i][0] / G[i] - 1), abs(m[i][1] / L[i] - 1)) for i in range(n)))
    return {"case": f"coexistence-curve-{n}-slabs-8x{ny}-Tr0.35-0.48-k0.2-mixed",
            "criterion": f"both bulks, averaged over {window} samples {every} steps apart, "
                         f"within {tol:g} of the method's equilibrium, every slab",
            "plain_sequential_tanh": {"wall_s": plain_s, "steps_per_slab": plain_steps,
                                      "all_reached": all(x is not None for x in plain_steps)},
            "batched_tanh": {"wall_s": batch_tanh_s, "steps": tanh_steps,
                             "reached": tanh_steps is not None},
            "batched_warm": {"wall_s": batch_s, "steps": steps, "reached": steps is not None,
                             "worst_windowed_rel_dev": worst},
            "speedup": plain_s / batch_s}


def warm_drop_case(s, eq, t_r, n=4096, radius=1000.0, every=5000, max_steps=100_000):
    """A 4096^2 drop of radius 1000 at T_r (k 0.2, kappa-hat 0.1, mixed), from the
    tanh start between the Maxwell densities and from the surrogate's warm start
    (its interface window mapped radially): steps until the bulk gas (the
    outermost 256 nodes of every side) and the bulk liquid (r < radius / 2) are
    both within 1e-3 of the long slab run's equilibrium eq, checked every
    `every` steps up to max_steps, and the deviations where the count stops.
    A drop of this size differs from the flat equilibrium by its Laplace
    pressure, far below 1e-3 in density."""
    import numpy as np
    import torch
    from paper_1906_09530_gb300 import LbmError, Simulation, lbm_maxwell, surrogate as SG
    from paper_1906_09530_gb300 import workloads as W
    rg, rl = lbm_maxwell(t_r)
    g, l, w = s.predict([t_r], [0.1], [0.2])
    yy, xx = torch.meshgrid(torch.arange(n, device="cuda", dtype=torch.float64),
                            torch.arange(n, device="cuda", dtype=torch.float64), indexing="ij")
    r = torch.hypot(xx - n / 2, yy - n / 2)
    liq = r < radius / 2
    b = 256
    gas = torch.zeros_like(liq)
    gas[:b, :] = gas[-b:, :] = gas[:, :b] = gas[:, -b:] = True

    def probe(sim):
        rho = sim.fields_device()[0]
        return float(rho[gas].mean()), float(rho[liq].mean())
    row = {"case": f"drop-{n}x{n}-R{int(radius)}-Tr{t_r}-k0.2-mixed", "checked_every": every,
           "max_steps": max_steps}
    for name, field in (("tanh", W.drop(n, n, rg, rl, radius, 20.0)),
                        ("warm", SG.drop_field(n, n, radius, g[0], l[0], w[0]))):
        sim = Simulation(n, n, t_r, 0.1, 1.0, 0.2, fd_order=6, precision="mixed")
        sim.set_fields(field)
        del field
        c0 = time.perf_counter()
        try:
            steps = SG.steps_to_equilibrium(sim, probe, eq, 1e-3, every=every,
                                            max_steps=max_steps)
        except LbmError as e:
            row[name] = {"error": str(e), "failed_step": sim.failed_step}
            sim.close()
            continue
        wall = time.perf_counter() - c0
        gv, lv = probe(sim)
        row[name] = {"steps_to_1e-3": steps, "wall_s": wall, "at_step": sim.t,
                     "gas_rel_dev": gv / eq[0] - 1, "liq_rel_dev": lv / eq[1] - 1}
        sim.close()
    return row


def drop_warm_start(train_T=(0.32, 0.33, 0.34, 0.36, 0.37, 0.38, 0.40),
                    radii=(64.0, 125.0, 250.0), judge_T=0.35, judge_R=250.0,
                    train_steps=300_000, run_steps=240_000, every=2000, window=10, kappa=0.1,
                    k=0.2, epochs=4000):
    """The learned warm start for drops: the 4096^2 drop of radius 1000 at T_r 0.35
    scaled down to a drop whose plain run converges (by default R 250 on 1000^2,
    the same grid/radius ratio).  Training data: drops of the given radii (each at the centre
    of a periodic grid 4 R wide) at the training temperatures, run as one batch
    for train_steps; the surrogate takes (T_r, kappa-hat, k, 1/R).  Judge: a drop
    of judge_R at judge_T (a temperature not trained on), from the tanh start
    between the Maxwell densities (the plain run, whose settled bulks are the
    target) and from the surrogate's prediction, its radius chosen so that the
    warm field holds the plain field's mass (the same system: a drop's
    equilibrium depends on its mass); each run samples the far-field
    gas (outer n/16 of every side) and the liquid core (r < R/2) every `every`
    steps, and its settling step is where the mean of the last `window` samples
    stays within 1e-3 of the target."""
    import numpy as np
    import torch
    from paper_1906_09530_gb300 import Simulation, lbm_maxwell, surrogate as SG
    from paper_1906_09530_gb300 import workloads as W
    T = np.repeat(np.asarray(train_T, dtype=np.float64), len(radii))
    R = np.tile(np.asarray(radii, dtype=np.float64), len(train_T))
    n = (4 * R).astype(int)
    t0 = time.perf_counter()
    G, L, P = SG.drop_profiles(T, np.full(T.size, kappa), np.full(T.size, k), R, n, train_steps)
    data_s = time.perf_counter() - t0
    s = SG.Surrogate(seed=7, ranges={"T_r": (min(train_T), max(train_T)),
                                     "kappa": (kappa, kappa), "k": (k, k)},
                     inv_r_range=(1.0 / max(radii), 1.0 / min(radii)), max_batch=256)
    t0 = time.perf_counter()
    loss = s.fit(T, np.full(T.size, kappa), np.full(T.size, k), G, L, P, epochs=epochs,
                 lr=2e-3, batch=T.size, inv_r=1.0 / R)
    fit_s = time.perf_counter() - t0
    g, l, w = s.predict([judge_T], [kappa], [k], inv_r=[1.0 / judge_R])
    s.close()
    m = int(4 * judge_R)
    rg, rl = lbm_maxwell(judge_T)
    yy, xx = torch.meshgrid(torch.arange(m, device="cuda", dtype=torch.float64),
                            torch.arange(m, device="cuda", dtype=torch.float64), indexing="ij")
    r = torch.hypot(xx - m / 2, yy - m / 2)
    liq = r < judge_R / 2
    b = m // 16
    gas = torch.zeros_like(liq)
    gas[:b, :] = gas[-b:, :] = gas[:, :b] = gas[:, -b:] = True
    runs = {}
    plain = W.drop(m, m, rg, rl, judge_R, 4.0 / k)
    # the warm start of the same system: its drop holds the plain start's mass
    warm_R = SG.drop_radius_for_mass(m, m, plain.sum(), g[0], l[0], w[0], judge_R)
    for name, field in (("plain", plain), ("warm", SG.drop_field(m, m, warm_R, g[0], l[0], w[0]))):
        sim = Simulation(m, m, judge_T, kappa, 1.0, k, fd_order=6, precision="mixed")
        sim.set_fields(field)
        times, samples, step_s = [], [], 0.0
        while True:
            rho = sim.fields_device()[0]
            times.append(sim.t)
            samples.append((float(rho[gas].mean()), float(rho[liq].mean())))
            if sim.t >= run_steps:
                break
            c0 = time.perf_counter()
            sim.step(every)  # returns when the steps are done
            step_s += time.perf_counter() - c0
        runs[name] = {"times": times, "samples": samples, "step_s": step_s}
        sim.close()
    # wall time of the stepping alone, per step, the same for both starts
    s_per_step = sum(rr["step_s"] for rr in runs.values()) / (2.0 * run_steps)
    target = np.mean(np.array(runs["plain"]["samples"][-window:]), axis=0)
    out = {"workload": f"drop-{m}x{m}-R{int(judge_R)}-Tr{judge_T}-k{k}-kappa{kappa}-mixed",
           "training": {"T_r": list(train_T), "radii": list(radii), "steps": train_steps,
                        "data_s": data_s, "fit_s": fit_s, "fit_loss": loss},
           "target_rel_maxwell": {"gas": target[0] / rg - 1, "liquid": target[1] / rl - 1},
           "predicted_rel_target": {"gas": g[0] / target[0] - 1, "liquid": l[0] / target[1] - 1},
           "warm_radius_same_mass": warm_R,
           "criterion": f"mean of the last {window} samples ({every} steps apart) within 1e-3 "
                        "of the plain run's settled bulks, and staying there"}
    for name, rr in runs.items():
        st = SG.settle_step(rr["times"], rr["samples"], target, 1e-3, window)
        v0 = np.array(rr["samples"][0])
        out[name] = {"settle_step": st, "wall_s_to_settle": (None if st is None else
                     s_per_step * st),
                     "start_rel_target": {"gas": v0[0] / target[0] - 1,
                                          "liquid": v0[1] / target[1] - 1},
                     "series_gas_rel_target": [round(x[0] / target[0] - 1, 5)
                                               for x in rr["samples"][::10]]}
    return out


def load_bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["bf16_tflops"]), "measured"
    return 1900.0, "fallback"


def max_over_ranks(seconds, dist, device):
    """The largest of every rank's elapsed time (seconds), on every rank; the
    job's time is its slowest replica's.  dist: torch.distributed or None."""
    if dist is None:
        return float(seconds)
    import torch
    t = torch.tensor([float(seconds)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(units_per_rank, world, seconds):
    """Whole-job throughput: the node updates of all ranks over the slowest
    rank's time, in millions per second."""
    return world * units_per_rank / seconds / 1e6


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import OracleSim, sim as S, thermo
    from paper_1906_09530_gb300 import workloads as W
    Tc, _ = thermo.critical_point()
    rg, rl = thermo.maxwell(w["T_r"])
    rho = W.drop(w["nx"], w["ny"], rg, rl, w["radius"], w["width"])
    # the oracle with its loops shared among all host cores (OpenMP)
    cores = S.set_threads(os.cpu_count() or 1)
    o = OracleSim(w["nx"], w["ny"], w["T_r"] * Tc, w["kappa"], w["tau"], w["k"], w["order"])
    o.set_fields(rho)
    # each reference step is one full-grid oracle step; up to three warm-up
    # steps, and the timed count bounded so that the run ends within about
    # three minutes
    warm = max(1, min(args.warmup, 3))
    t0 = time.perf_counter()
    o.step(1)
    per = time.perf_counter() - t0
    budget = 150.0
    k = max(1, min(args.steps, int(budget / max(per, 1e-6))))
    if warm > 1:
        o.step(warm - 1)
    t0 = time.perf_counter()
    o.step(k)
    dt = time.perf_counter() - t0
    N = w["nx"] * w["ny"]
    val = N * k / dt / 1e6
    line = {"metric": METRIC, "value": val, "unit": "MLUPS", "impl": "reference",
            "n_gpus": args.gpus, "steps": k, "warmup": warm, "ms_per_step": dt / k * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(w, args.precision),
                       "arithmetic": "the FP64 oracle on the same workload"},
            "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"{k} full-grid FP64 oracle step{'s' * (k != 1)} "
                                       f"(of {args.steps} asked; bounded to ~150 s), "
                                       f"{cores} threads (OpenMP over lines and nodes)"},
            "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--size", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-equilibrium", action="store_true")
    ap.add_argument("--surrogate", action="store_true",
                    help="add the learned warm start's measurement (several minutes)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the collide-stream form comparison")
    ap.add_argument("--no-mlp", action="store_true",
                    help="skip the surrogate network's product timings")
    ap.add_argument("--mlp-batches", default="256,4096,32768",
                    help="batch sizes of the network timings (comma-separated)")
    ap.add_argument("--mlp-reps", type=int, default=50)
    ap.add_argument("--surrogate-drop", action="store_true",
                    help="add the learned warm start for drops (a few minutes)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched-instances line")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 4096^2 line (default: measured after the main one)")
    ap.add_argument("--no-splash", action="store_true",
                    help="skip the drop-splashing lines (walls; 2048 x 1024 and the "
                         "paper's 1000 x 300)")
    args = ap.parse_args()
    w = dict(WORKLOAD)
    if args.size != 1024:
        s = args.size / 1024
        w.update(nx=args.size, ny=args.size, radius=w["radius"] * s)
    if args.impl == "reference":
        return run_reference(args, w)
    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps")

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_1906_09530_gb300 as P
    from paper_1906_09530_gb300 import workloads as W
    rg, rl = P.lbm_maxwell(w["T_r"])
    rho0 = W.drop(w["nx"], w["ny"], rg, rl, w["radius"], w["width"])
    N = w["nx"] * w["ny"]
    sim = P.Simulation(w["nx"], w["ny"], w["T_r"], w["kappa"], w["tau"], w["k"],
                       fd_order=w["order"], precision=args.precision)
    sim.set_fields(rho0)
    sim.step(args.warmup)
    # L2 flush between timed steps: write 512 MB (evicts the simulation's data),
    # then read another 512 MB so that L2 holds clean lines and the step does not
    # pay for writing back the flush buffer's dirty lines
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    clean = torch.zeros(128 << 20, dtype=torch.float32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(bus_id(local))
    barrier()
    names, pb = pass_layout(args.precision, sim.path_flags)
    # the timed region: K steps, each bracketed by one CUDA event pair on the
    # library's stream, with the L2 flushed between them (not timed)
    ev_a = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_b = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        clean.amax()
        ev_a[i].record()
        sim.step_async(1)
        ev_b[i].record()
    barrier()
    clk = clocks.stop()
    sim.check()
    step_ms = np.array([a.elapsed_time(b) for a, b in zip(ev_a, ev_b)])
    total_s = max_over_ranks(step_ms.sum() / 1e3, dist, "cuda")
    value = whole_job_mlups(N * args.steps, world, total_s)
    # the per-pass breakdown (after the timed region): events around every pass
    npass = min(args.steps, 200)
    pass_ms = np.zeros((npass, 5))
    for i in range(npass):
        flush.zero_()
        clean.amax()
        pass_ms[i] = sim.step_timed()
    pass_ms = pass_ms[:, :len(names)]

    # back-to-back CUDA-graph steps without flushing (context only)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kb = max(2, args.steps // 2 * 2)
    torch.cuda.synchronize()
    ev0.record()
    sim.step_async(kb)
    ev1.record()
    sim.check()
    graph_mlups = N * kb / (ev0.elapsed_time(ev1) / 1e3) / 1e6

    # e2e through the public host API, pinned host buffers
    e2e = None
    if not args.no_e2e:
        h_rho = torch.from_numpy(rho0).pin_memory().numpy()
        outs = [torch.empty((w["ny"], w["nx"]), dtype=torch.float64).pin_memory().numpy()
                for _ in range(4)]
        from paper_1906_09530_gb300._binding import _check, _hptr, lib
        barrier()
        t0 = time.perf_counter()
        _check(lib().lbm_set_fields(sim.ctx, _hptr(h_rho), None, None), "lbm_set_fields")
        _check(lib().lbm_step(sim.ctx, args.steps), "lbm_step")
        _check(lib().lbm_fields(sim.ctx, *[_hptr(a) for a in outs]), "lbm_fields")
        dt = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        e2e = {"value": whole_job_mlups(N * args.steps, world, dt), "unit": "MLUPS",
               "h2d_bytes_per_step": N * 8 / args.steps,
               "d2h_bytes_per_step": 4 * N * 8 / args.steps,
               "what": "lbm_set_fields(host rho) + lbm_step(K) + lbm_fields(rho, vx, vy, "
                       "mu to host), wall clock; bytes per step = run totals / K"}

    mean_pass = pass_ms.mean(axis=0)
    peak, peak_kind = load_peaks()
    dom = int(np.argmax(mean_pass))
    passes = {}
    for i, nm in enumerate(names):
        gbs = pb[i] * N / (mean_pass[i] / 1e3) / 1e9
        passes[nm] = {"ms": round(float(mean_pass[i]), 5), "alg_bytes_per_node": pb[i],
                      "GB/s": round(gbs, 1), "frac_hbm": round(gbs / peak, 4)}
    ach = pb[dom] * N / (mean_pass[dom] / 1e3) / 1e9
    tr = measured_traffic(args.precision)
    roofline = {"bound": "hbm", "kernel": names[dom], "achieved": ach, "peak": peak,
                "unit": "GB/s", "frac": ach / peak,
                "traffic": None if tr is None or names[dom] not in tr else tr[names[dom]] * N,
                "peak_kind": f"{peak_kind} copy bandwidth",
                "alg_bytes_per_launch": pb[dom] * N}
    step_gbs = sum(pb) * N / (float(step_ms.mean()) / 1e3) / 1e9
    roofline["frac_nominal"] = ach / HBM_NOMINAL_GBS
    roofline["step"] = {"alg_bytes_per_node": sum(pb), "achieved": step_gbs,
                        "frac": step_gbs / peak, "frac_nominal": step_gbs / HBM_NOMINAL_GBS,
                        "what": "whole step: the algorithmic bytes of all its passes over "
                                "the mean step time; frac against the measured copy peak, "
                                "frac_nominal against 7.9 TB/s"}
    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(step_ms.mean()), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(w, args.precision), "nodes": N,
                       "l2": "512 MB write + 512 MB read between timed steps "
                             "(L2 flushed, left clean)",
                       "parallelism": f"replicas{world}" if world > 1 else "single"},
            "roofline": roofline,
            "step_roofline": {"alg_bytes_per_node": sum(pb), "achieved_GB/s": step_gbs,
                              "frac": step_gbs / peak,
                              "frac_at_216B_fp64_field_convention":
                                  216 * N / (float(step_ms.mean()) / 1e3) / 1e9 / peak},
            "passes": passes,
            "graph_back_to_back_mlups": graph_mlups,
            "e2e": e2e, "gpu_launches": len(names) * args.steps, "clocks": clk}
    if not args.no_large and args.size < 4096:
        lg = large_grid(args.precision, min(args.steps, 100), max(args.warmup, 3))
        line["large_grid"] = lg
        # the same figures at 4096^2, where the working set is far above L2
        sr = lg["step_roofline"]
        roofline["at_4096"] = {
            "workload": lg["workload"], "mlups": lg["mlups"],
            "kernel": lg["dominant"]["kernel"], "achieved": lg["dominant"]["achieved_GB/s"],
            "frac": lg["dominant"]["frac"],
            "frac_nominal": lg["dominant"]["achieved_GB/s"] / HBM_NOMINAL_GBS,
            "passes_frac": lg["passes_frac_hbm"],
            "step_achieved": sr["achieved_GB/s"], "step_frac": sr["frac"],
            "step_frac_nominal": sr["achieved_GB/s"] / HBM_NOMINAL_GBS}
        # MRT with the paper's rates is unstable on the T_r 0.5, k 0.5 drop
        # (as in the oracle); its throughput is taken on a stable T_r 0.7, k 0.3 one
        line["large_grid_mrt"] = large_grid(args.precision, min(args.steps, 100),
                                            max(args.warmup, 3), collision="mrt", T_r=0.7,
                                            k=0.3, width=4.0 / 0.3)
        # the same drop at 8192^2 (about 7 GB of workspace), and the FP64 path at 4096^2
        line["large_grid_8192"] = large_grid(args.precision, min(args.steps, 50),
                                             max(args.warmup, 3), size=8192)
        if args.precision != "fp64":
            line["large_grid_fp64"] = large_grid("fp64", min(args.steps, 20),
                                                 max(args.warmup, 3), size=4096)
            line["fp64_path"] = fp64_path_summary(line["large_grid_fp64"])
    if not args.no_batch and args.precision == "mixed":
        line["batch"] = batch_config(min(args.steps, 50), max(args.warmup // 10, 3))
    if rank == 0 and not args.no_splash:
        line["splash"] = splash_config(args.precision)
        line["splash_paper"] = splash_paper_config()
    if rank == 0 and not args.no_forms and args.precision == "mixed":
        line["collide_forms"] = collide_forms()
        line["launch_overlap"] = launch_overlap()
    if rank == 0 and not args.no_mlp:
        line["mlp"] = mlp_products(tuple(int(b) for b in args.mlp_batches.split(",")),
                                   args.mlp_reps)
    if rank == 0 and args.surrogate:
        line["surrogate"] = surrogate_demo()
    if rank == 0 and args.surrogate_drop:
        line["surrogate_drop"] = drop_warm_start()
    if rank == 0 and not args.no_equilibrium:
        line["equilibrium"] = equilibrium_time(args.precision)
        # the same slab 1024 nodes wide (409 600 nodes, the grid scale of the
        # benchmark drop)
        line["equilibrium_1024"] = equilibrium_time(args.precision, nx=1024)
        # the lowest temperature at which the method's gas comes within 1e-3 of
        # Maxwell at k 0.1
        line["equilibrium_0.7"] = equilibrium_time(args.precision, T_r=0.7)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    sim.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
