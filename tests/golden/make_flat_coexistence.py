"""Writes flat_coexistence.json: the converged bulk densities of flat periodic
slabs under the method as the oracle reads it (Sec. 5.1's set-up: a 1-D domain
with two planar interfaces, k = 0.1 and height 400 unless varied, CS EOS with
a = 1, b = 4, R = 1, tau = 1, 6th-order compact scheme), found by the oracle's
direct equilibrium solver.  Calls only oracle/.  Run from the repository root:
    python tests/golden/make_flat_coexistence.py
(about 40 minutes; the dilute gas below T_r ~ 0.25 is finished by time
stepping, see oracle/equilibrium.py).

With --redo T_r k [T_r k ...] it recomputes those entries only.  With
--fixed-points it writes flat_fixed_points.json instead: the whole
converged state (the six reduced populations per node, oracle/equilibrium.py)
of the height-400, k = 0.1 slab at T_r 0.3 and 0.2, from which GPU tests start.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import equilibrium as E  # noqa: E402
from oracle import sim as S  # noqa: E402

KAPPA, TAU = 0.1, 1.0


def entry(T_r, k, n):
    r = E.flat_equilibrium(n, T_r, KAPPA, TAU, k, steps=20000)
    rg, rl = r["maxwell"]
    return {"T_r": T_r, "k": k, "height": n, "rho_g": r["rho_g"], "rho_l": r["rho_l"],
            "maxwell_g": rg, "maxwell_l": rl, "gas_offset": r["gas_offset"],
            "liq_offset": r["liq_offset"], "gas_offset_decades": r["log10_gas_offset"],
            "newton_residual": r["residual"], "relative_residual": r["relative_residual"],
            "polish_steps": r["polish_steps"]}


def main():
    S.set_threads(4)  # the C oracle's time stepping (same bits on any thread count)
    out = {"_what": "Converged flat-slab bulk densities of the method (oracle/equilibrium.py), "
                    "against the Maxwell pair; kappa-hat 0.1, tau 1, CS a=1 b=4 R=1, 6th order. "
                    "Written by tests/golden/make_flat_coexistence.py from oracle/ only.",
           "curve_k0.1": [], "k_series": []}
    for T_r in (0.8, 0.7, 0.6, 0.5, 0.45, 0.4, 0.35, 0.3, 0.25, 0.2, 0.16):
        out["curve_k0.1"].append(entry(T_r, 0.1, 400))
        print(out["curve_k0.1"][-1], flush=True)
    for T_r in (0.6, 0.4, 0.3, 0.2, 0.16):
        for k in (0.4, 0.2, 0.1, 0.05):
            if T_r <= 0.3 and k > 0.1:
                continue
            out["k_series"].append(entry(T_r, k, int(round(40 / k))))
            print(out["k_series"][-1], flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "flat_coexistence.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)


def fixed_points():
    S.set_threads(4)
    out = {"_what": "Converged states of the flat slab (height 400, k 0.1, kappa-hat 0.1, "
                    "tau 1, CS a=1 b=4 R=1, 6th order): the six reduced populations "
                    "g0, gx, gu, gd, gux, gdx per node (oracle/equilibrium.py). Written by "
                    "tests/golden/make_flat_coexistence.py --fixed-points from oracle/ only.",
           "states": []}
    for T_r in (0.3, 0.2):
        r = E.flat_equilibrium(400, T_r, KAPPA, TAU, 0.1, steps=20000)
        out["states"].append({"T_r": T_r, "k": 0.1, "height": 400,
                              "relative_residual": r["relative_residual"],
                              "g": [[float(v) for v in row] for row in r["g"]]})
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "flat_fixed_points.json")
    with open(path, "w") as fh:
        json.dump(out, fh)


def redo(pairs):
    """Recompute the entries (T_r, k) given and update flat_coexistence.json."""
    S.set_threads(4)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "flat_coexistence.json")
    out = json.load(open(path))
    for key in ("curve_k0.1", "k_series"):
        for i, e in enumerate(out[key]):
            if (e["T_r"], e["k"]) in pairs:
                out[key][i] = entry(e["T_r"], e["k"], e["height"])
                print(out[key][i], flush=True)
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    if "--fixed-points" in sys.argv:
        fixed_points()
    elif "--redo" in sys.argv:
        v = [float(x) for x in sys.argv[sys.argv.index("--redo") + 1:]]
        redo(set(zip(v[0::2], v[1::2])))
    else:
        main()
