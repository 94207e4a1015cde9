"""The mixed path's two collide-stream forms (lbm_set_collide_form): the
row-ring kernel (16-byte asynchronous copies of 128-column row pieces into a
shared-memory ring) and the sliding-window kernel (three rows in registers, warp
shuffles) collide and stream with the same rounded arithmetic, so populations and
the density pair must agree bit for bit after any number of steps.  Grids cover one and
several 120-column strips with a ragged last strip, the smallest width the
ring takes (128), rows segments with a ragged tail, both wraps in x and y, MRT,
and the grids where the ring does not apply (walls, nx not a multiple of 4,
nx < 128), which must fall back to the sliding window."""
import numpy as np
import pytest

from paper_1906_09530_gb300 import Simulation, lbm_maxwell
from paper_1906_09530_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RING = 4  # LBM_PATH_CS_RING


def _pair(nx, ny, T_r=0.5, k=0.5, collision="bgk", walls_y=False, rows=8, steps=7):
    rg, rl = lbm_maxwell(T_r)
    # centred, so the tanh tails meet the periodic seams symmetrically
    rho = W.drop(nx, ny, rg, rl, 0.25 * min(nx, ny), 4.0 / k)
    out = []
    for form in (rows, -1):
        s = Simulation(nx, ny, T_r, 0.1, 1.0, k, fd_order=6, precision="mixed",
                       collision=collision, walls_y=walls_y)
        s.set_collide_form(form)
        s.set_fields(rho)
        s.step(steps)
        f, t = s.get_populations()
        out.append((f, s.fields()[0], s.path_flags))
        s.close()
    return out


@pytest.mark.parametrize("nx,ny", [(1024, 1024), (128, 96), (132, 77), (360, 41),
                                   (484, 300), (1000, 33)])
def test_ring_matches_sliding_window(cuda, nx, ny):
    (f_r, rho_r, fl_r), (f_s, rho_s, fl_s) = _pair(nx, ny)
    assert fl_r & RING and not fl_s & RING
    assert np.array_equal(f_r, f_s)
    assert np.array_equal(rho_r, rho_s)


@pytest.mark.parametrize("rows", [1, 3, 8, 16, 32, 200])
def test_ring_rows_per_block(cuda, rows):
    """Any rows-per-block choice gives the same bits (ragged last segment,
    a segment of one row, a segment taller than the grid)."""
    (f_r, _, fl_r), (f_s, _, _) = _pair(256, 150, rows=rows)
    assert fl_r & RING
    assert np.array_equal(f_r, f_s)


def test_ring_mrt(cuda):
    (f_r, _, fl_r), (f_s, _, _) = _pair(248, 64, T_r=0.7, k=0.3, collision="mrt")
    assert fl_r & RING
    assert np.array_equal(f_r, f_s)


@pytest.mark.parametrize("nx,ny,walls", [(130, 64, False), (124, 64, False), (256, 64, True)])
def test_ring_falls_back(cuda, nx, ny, walls):
    """nx not a multiple of 4, nx < 128, or walls: the sliding window runs."""
    (f_r, _, fl_r), (f_s, _, _) = _pair(nx, ny, walls_y=walls)
    assert not fl_r & RING
    assert np.array_equal(f_r, f_s)


@pytest.mark.parametrize("n,ring", [(1024, False), (2048, False), (4096, True)])
def test_default_form_by_size(cuda, n, ring):
    """The default (0) takes the sliding window below 2^23 nodes and the ring at
    and above, where each is the faster."""
    s = Simulation(n, n, 0.5, 0.1, 1.0, 0.5, fd_order=6, precision="mixed")
    assert bool(s.path_flags & RING) == ring
    s.set_collide_form(8)
    assert s.path_flags & RING
    s.set_collide_form(-1)
    assert not s.path_flags & RING
    s.close()


def test_ring_long_run_against_oracle_parity_size(cuda):
    """The ring at the benchmark's 1024^2 drop stays bit-identical to the sliding
    window over 200 steps (the oracle parity tests at this size run the sliding
    window, the default there)."""
    (f_r, rho_r, fl_r), (f_s, rho_s, _) = _pair(1024, 1024, steps=200)
    assert fl_r & RING
    assert np.array_equal(f_r, f_s)


@pytest.mark.parametrize("mode", [(0, 0, 0), (0, 1, 0), (0, 1, 1), (1, 0, 0), (1, 0, 1)])
def test_launch_mode_keeps_results(cuda, mode):
    """Graph or direct lone steps and programmatic dependent launch change when
    the kernels are scheduled, not what they compute: single steps and graph
    replays give the default setting's populations bit for bit."""
    rg, rl = lbm_maxwell(0.5)
    rho = W.drop(512, 384, rg, rl, 96.0, 8.0)
    out = []
    for m in ((1, 1, 0), mode):
        s = Simulation(512, 384, 0.5, 0.1, 1.0, 0.5, fd_order=6, precision="mixed")
        s.set_launch_mode(*m)
        s.set_fields(rho)
        for _ in range(3):
            s.step_async(1)  # lone steps
        s.step(21)           # graph replays and an odd last step
        out.append(s.get_populations()[0])
        s.close()
    assert np.array_equal(out[0], out[1])
