"""The 1024 x 1024 static drop of radius 200 (k = 0.5, kappa-hat 0.1, tau 1,
6th-order compact scheme, tanh width 8) at T_r 0.6, 0.5 and 0.45 (Maxwell
density ratios 132, 725 and 2327), 20 000 steps, run by the FP64 path and by
the mixed path (FP32 populations and collision, the density as an exact
double-float pair, compact derivatives of the density in FP32 below a ratio of
1e4) and the mixed path with double-float density lines throughout
("mixed_df").  The FP64 path is the reference (it follows the oracle to 1e-10
over 1000 steps in test_gpu_parity.py); each mixed result is compared with it
node by node and by its bulk densities:
  * liquid: the mean over r < R/2;
  * gas: the mean over nodes farther than R + 60 from the drop's centre
    (periodic distance), outside the interface's tail.
After 20 000 steps the drop is still relaxing (its acoustic waves and the slow
gas diffusion), so node by node the largest relative differences sit in the
interface's gas-side tail, where a shift of the profile by a small fraction of
a node changes the local density by percents; there the difference is also
stated relative to the density jump rho_l - rho_g.
Measured on one GB300 (the largest of the three temperatures, mixed and
mixed_df alike): bulk gas 8.9e-5, bulk liquid 1.6e-5, any node 2.7e-2
relative to itself and 8.0e-3 of the density jump.  The bounds are about twice
those.
"""
import numpy as np
import pytest

from tests import cases

pytestmark = pytest.mark.gpu

STEPS = 20_000
# measured (one GB300): the largest errors of the three temperatures
BOUNDS = {"node": 5e-2, "node_jump": 1.6e-2, "gas": 2e-4, "liquid": 4e-5}


def _bulks(rho, radius):
    n = rho.shape[0]
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    dx = np.minimum(np.abs(x - n / 2), n - np.abs(x - n / 2))
    dy = np.minimum(np.abs(y - n / 2), n - np.abs(y - n / 2))
    r = np.hypot(dx, dy)
    return float(rho[r > radius + 60].mean()), float(rho[r < radius / 2].mean())


@pytest.fixture(scope="module")
def runs(cuda):
    out = {}
    for T_r in (0.6, 0.5, 0.45):
        c = cases.config2(T_r)
        for prec in ("fp64", "mixed", "mixed_df"):
            s = cases.gpu_sim(c, precision=prec)
            s.set_fields(c["rho"])
            s.step(STEPS)
            out[T_r, prec] = s.fields()[0]
            s.close()
    return out


@pytest.mark.parametrize("prec", ["mixed", "mixed_df"])
@pytest.mark.parametrize("T_r", [0.6, 0.5, 0.45])
def test_drop_1024_mixed_against_fp64(runs, T_r, prec):
    ref, got = runs[T_r, "fp64"], runs[T_r, prec]
    node = float(np.abs(got / ref - 1).max())
    g_ref, l_ref = _bulks(ref, 200.0)
    g, l = _bulks(got, 200.0)
    jump = float(np.abs(got - ref).max() / (l_ref - g_ref))
    gas, liq = abs(g / g_ref - 1), abs(l / l_ref - 1)
    print(f"\n1024^2 drop T_r {T_r} {prec} vs fp64 after {STEPS} steps: node {node:.3e} "
          f"node/jump {jump:.3e} gas {gas:.3e} liquid {liq:.3e} "
          f"(fp64 bulks {g_ref:.6e} {l_ref:.6e})")
    b = BOUNDS
    assert node <= b["node"] and jump <= b["node_jump"], (node, jump)
    assert gas <= b["gas"] and liq <= b["liquid"], (gas, liq)
