"""Seeded synthetic initial fields for the benchmark and the tests.

This module holds no arithmetic of the method itself: it only lays out initial
density and velocity fields (numpy, FP64, row-major [ny][nx]) from coexistence
densities that the caller supplies.  Both the CUDA path and the CPU oracle are
fed from here, so their inputs are bit-identical.

  * drop      the tanh profile of Eq. 41 around the domain centre
  * flat      two planar interfaces normal to y, liquid in the middle (Sec. 5.1)
  * noise     multiplicative uniform noise rho <- rho (1 + eps), eps in [-A, A],
              drawn from splitmix64 of (seed, node index): a counter-based
              generator, so any node's value can be recomputed on its own.
  * batch     a seeded set of many independent instances (uneven grid sides and
              temperatures, drops and flat interfaces) for the batched path.
  * splash    a liquid film on the bottom wall and a drop falling onto it
              (Sec. 5.5), with an optional uniform shift of the reference frame.
"""
import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x):
    """splitmix64 finaliser (Steele, Lea and Flood, 2014) on a uint64 array."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def uniform_noise(shape, seed, amplitude):
    """eps in [-amplitude, amplitude) for every node, node index = y*nx + x."""
    n = int(np.prod(shape))
    idx = np.arange(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        key = splitmix64(np.uint64(seed) * np.uint64(0x100000001B3) + idx)
    u = (key >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)  # [0,1)
    return (amplitude * (2.0 * u - 1.0)).reshape(shape)


def drop(nx, ny, rho_g, rho_l, radius, width, center=None):
    """Eq. 41: rho = (rho_g+rho_l)/2 + (rho_g-rho_l)/2 tanh(2(r - r0)/W), centre
    (nx/2, ny/2) in node indices unless given."""
    x0, y0 = (nx / 2.0, ny / 2.0) if center is None else center
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.sqrt((x - x0) ** 2 + (y - y0) ** 2)
    return 0.5 * (rho_g + rho_l) + 0.5 * (rho_g - rho_l) * np.tanh(2.0 * (r - radius) / width)


def flat(nx, ny, rho_g, rho_l, thickness, width):
    """Liquid slab |y - ny/2| < thickness/2 in gas, tanh edges of width W."""
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    d = np.abs(y - ny / 2.0) - thickness / 2.0
    return 0.5 * (rho_g + rho_l) + 0.5 * (rho_g - rho_l) * np.tanh(2.0 * d / width)


def with_noise(rho, seed, amplitude):
    """Multiplicative noise, rho (1 + eps): keeps low gas densities positive."""
    return rho * (1.0 + uniform_noise(rho.shape, seed, amplitude))


def shear_wave(nx, ny, rho0, amplitude):
    """Uniform density with u_x = A sin(2 pi y / ny), u_y = 0."""
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    return (np.full((ny, nx), rho0), amplitude * np.sin(2 * np.pi * y / ny),
            np.zeros((ny, nx)))


BATCH_SIDES = (64, 128, 256, 512)


def batch_instances(n=256, seed=1234, t_lo=0.3, t_hi=0.9):
    """n independent periodic instances: square grids with sides drawn uniformly
    from BATCH_SIDES (splitmix64 of (seed, i)), T_r log-spaced from t_lo to t_hi,
    each a drop of radius side/4 or a flat slab of thickness side/2 (again from
    splitmix64).  k = 0.5 for T_r >= 0.45 and 0.3 below (k = 0.5 drops blow up at
    T_r <= 0.4), kappa-hat = 0.1, tau = 1, tanh width 4/k."""
    idx = np.arange(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        key = splitmix64(np.uint64(seed) * np.uint64(0x100000001B3) + idx)
    sides = [BATCH_SIDES[int(v)] for v in (key >> np.uint64(40)) % np.uint64(len(BATCH_SIDES))]
    kinds = ["drop" if int(v) else "flat" for v in (key >> np.uint64(20)) & np.uint64(1)]
    trs = np.geomspace(t_lo, t_hi, n) if n > 1 else np.array([t_lo])
    out = []
    for i in range(n):
        k = 0.5 if trs[i] >= 0.45 else 0.3
        out.append(dict(nx=sides[i], ny=sides[i], T_r=float(trs[i]), k=k, kappa=0.1, tau=1.0,
                        kind=kinds[i], width=4.0 / k))
    return out


def batch_field(spec, rho_g, rho_l):
    """Initial density of one batch instance from its coexistence pair."""
    n = spec["nx"]
    if spec["kind"] == "drop":
        return drop(spec["nx"], spec["ny"], rho_g, rho_l, 0.25 * n, spec["width"])
    return flat(spec["nx"], spec["ny"], rho_g, rho_l, 0.5 * spec["ny"], spec["width"])


def splash(nx, ny, rho_g, rho_l, film, radius, height, width, u_drop, u_shift=0.0):
    """(rho, ux, uy): a film of thickness `film` on the bottom wall (rows 0 ..)
    and a drop of the given radius whose centre is `height` above the film's
    surface, at x = nx/2, moving at uy = u_drop; tanh edges of width W (Eq. 41).
    u_shift adds a uniform ux everywhere (a moving reference frame)."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    film_phi = 0.5 * (1.0 - np.tanh(2.0 * (y - film) / width))
    r = np.sqrt((x - nx / 2.0) ** 2 + (y - film - height) ** 2)
    drop_phi = 0.5 * (1.0 - np.tanh(2.0 * (r - radius) / width))
    phi = np.maximum(film_phi, drop_phi)
    rho = rho_g + (rho_l - rho_g) * phi
    return rho, np.full_like(rho, u_shift), u_drop * drop_phi
