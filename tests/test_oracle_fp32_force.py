"""Why the mixed path's FP32 force takes c_s^2 = 1/3 as a pair hi + lo rounded
once (Eq. 12), and not as the FP32 constant 1/3, which is 3.0e-8 too large.

The check runs on the oracle's flat slab of Sec. 5.1 (k 0.1, height 400, kappa-hat
0.1, tau 1, 6th-order CFD) at T_r 0.3, where the method's own equilibrium has a
density ratio of 1e6. It starts on the oracle's fixed point of the step
(tests/golden/flat_fixed_points.json) and holds the populations in FP32 after
every step. Everything is the oracle's FP64 arithmetic except the force's last
operation, F = -rho d(mu-hat) + c_s^2 d(rho), which is restated in FP32 the two
ways below. An FMA is restated as an FP64 product and sum rounded once to FP32:
the product of two FP32 values is exact in FP64.

  * c_s^2 = float32(1/3): F = fma(-rho, d mu, d rho * c).  Against the
    populations' exact 1/3, the bias is a spurious force at the interface; through
    grad(mu-hat) = c_s^2 grad(ln rho) in the gas it shifts the dilute gas,
    measured at -4.2e-4 after 20 000 steps.
  * c_s^2 = hi + lo: F = fma(d rho, hi, fma(-rho, d mu, d rho * lo)).  The gas
    stays within 1.2e-7, near the 3e-10 of FP32 storage alone.

It calls no library code.
"""
import json
import os

import numpy as np

from oracle import equilibrium as E

f32 = np.float32
STEPS = 20_000


def _fma32(a, b, c):
    return (a.astype(np.float64) * np.float64(b) + c.astype(np.float64)).astype(f32)


class _Fp32ForceSlab(E.FlatSlab):
    """The oracle's slab with the force's last operation in FP32."""

    def __init__(self, split, *args):
        super().__init__(*args)
        self.split = split

    def force(self, rho):
        d_rho = self.D @ rho
        mu = self.k ** 2 * self.eos.mu0(rho, self.T, self.al) - self.kappa * (self.D @ d_rho)
        r, dmu, d = rho.astype(f32), (self.D @ mu).astype(f32), d_rho.astype(f32)
        if self.split:
            hi = f32(1.0 / 3.0)
            lo = f32(1.0 / 3.0 - float(hi))
            F = _fma32(d, hi, _fma32(-r, dmu, d * lo))
        else:
            F = _fma32(-r, dmu, d * f32(1.0 / 3.0))
        return mu, F.astype(np.float64)


def _gas_shift(split):
    p = os.path.join(os.path.dirname(__file__), "golden", "flat_fixed_points.json")
    st = next(s for s in json.load(open(p))["states"] if s["T_r"] == 0.3)
    g = np.array(st["g"])
    slab = _Fp32ForceSlab(split, st["height"], 0.3, 0.1, 1.0, st["k"], 6)
    rho0 = slab.moments(g)[0]
    far = int(np.argmin(rho0))  # the gas node farthest from both interfaces
    g = g.astype(f32).astype(np.float64)
    for _ in range(STEPS):
        g = slab.step(g).astype(f32).astype(np.float64)
    return slab.moments(g)[0][far] / rho0[far] - 1


def test_split_constants_are_one_third():
    hi = f32(1.0 / 3.0)
    lo = f32(1.0 / 3.0 - float(hi))
    assert float(hi) / (1.0 / 3.0) - 1 > 2.9e-8          # the FP32 constant's bias
    assert abs(float(hi) + float(lo) - 1.0 / 3.0) < 1e-15


def test_fp32_force_with_the_rounded_constant_moves_the_gas():
    assert _gas_shift(False) < -1e-4


def test_fp32_force_with_split_constant_holds_the_gas():
    assert abs(_gas_shift(True)) < 1e-6
