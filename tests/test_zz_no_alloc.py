"""lbm_diag_noalloc: the diagnostics computed with the reduction's scratch in the
library's own fixed device array, for callers that cannot allocate device
memory.  Called through the C ABI and checked against lbm_diag (whose scratch is
in the caller's workspace) on two calls in a row, at the tolerances the other
diagnostics tests use.  Kept in the last-collected file so that a run that stops
at the first failure has already run everything else.
"""
import ctypes as C

import numpy as np
import pytest

from tests import cases

pytestmark = pytest.mark.gpu


def _diag(fn, sim):
    v = [C.c_double() for _ in range(4)]
    st = fn(sim.ctx, *[C.byref(x) for x in v])
    assert st == 0, st
    return [x.value for x in v]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_diag_noalloc_matches_diag(cuda, precision):
    from paper_1906_09530_gb300 import lib
    c = cases.ragged(nx=200, ny=168)
    sim = cases.gpu_sim(c, precision=precision)
    sim.set_fields(c["rho"])
    for _ in range(2):
        sim.step(7)
        ref = _diag(lib().lbm_diag, sim)
        got = _diag(lib().lbm_diag_noalloc, sim)
        assert got[0] == pytest.approx(ref[0], rel=1e-13)
        assert got[1] == pytest.approx(ref[1], rel=1e-12)
        assert got[2] == ref[2] and got[3] == ref[3]
        rho = sim.fields()[0]
        assert got[0] == pytest.approx(rho.sum(), rel=1e-13)
    sim.close()


def test_diag_noalloc_rejects_oversize_grid(cuda):
    """Grids above the fixed array's capacity (33,554,432 nodes) are refused
    before any device work."""
    from paper_1906_09530_gb300 import Simulation, lib
    from paper_1906_09530_gb300._binding import LBM_EINVAL
    sim = Simulation(8192, 4104, 0.6, 0.1, 1.0, 0.5, fd_order=6, precision="mixed")
    sim.set_fields(np.full((4104, 8192), 0.2))
    v = [C.c_double() for _ in range(4)]
    assert lib().lbm_diag_noalloc(sim.ctx, *[C.byref(x) for x in v]) == LBM_EINVAL
    sim.close()
