"""ctypes front end of the C oracle (cplbm_oracle.c).

TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the benchmark's
CPU-baseline leg use this module.  It never touches the CUDA library.

Arrays are numpy float64, C-contiguous, row-major [ny][nx]; populations are
structure-of-arrays [9][ny][nx] in the velocity order of Sec. 2.
"""
import ctypes as C
import math

import numpy as np

from . import build as _build

_lib = None


class OrcParams(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32),
                ("T", C.c_double), ("a", C.c_double), ("b", C.c_double),
                ("R", C.c_double),
                ("kappa", C.c_double), ("tau", C.c_double), ("k", C.c_double),
                ("alpha", C.c_double),
                ("mu_max", C.c_double), ("mu_cap_steps", C.c_int64),
                ("eos", C.c_int32), ("eos_alpha", C.c_double),
                ("mrt", C.c_int32), ("s", C.c_double * 9), ("walls_y", C.c_int32),
                ("wall_ux", C.c_double * 2)]

# MRT relaxation rates of Sec. 2 (after Eq. 4): s_e, s_eps, s_q; s_v = 1/tau
PAPER_MRT = (1.64, 1.54, 1.9)

# EOS kinds of the C oracle (its header comment)
EOS_KIND = {"cs": 0, "vdw": 1, "rk": 2, "rks": 3, "pr": 4}


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        dp = C.POINTER(C.c_double)
        P = C.POINTER(OrcParams)
        L.orc_cs_p0.restype = C.c_double
        L.orc_cs_p0.argtypes = [C.c_double] * 5
        L.orc_cs_mu0.restype = C.c_double
        L.orc_cs_mu0.argtypes = [C.c_double] * 5
        L.orc_cfd_field.restype = C.c_int
        L.orc_cfd_field.argtypes = [P, C.c_int, dp, dp]
        L.orc_mrt_matrices.restype = None
        L.orc_mrt_matrices.argtypes = [dp, dp]
        L.orc_p0.restype = C.c_double
        L.orc_p0.argtypes = [C.c_int] + [C.c_double] * 6
        L.orc_mu0.restype = C.c_double
        L.orc_mu0.argtypes = [C.c_int] + [C.c_double] * 6
        L.orc_cfd_line.restype = C.c_int
        L.orc_cfd_line.argtypes = [dp, C.c_ssize_t, dp, C.c_ssize_t, C.c_int,
                                   C.c_double, C.c_double]
        L.orc_forcing_terms.restype = None
        L.orc_forcing_terms.argtypes = [C.c_double] * 5 + [dp]
        L.orc_feq_field.restype = None
        L.orc_feq_field.argtypes = [P, dp, dp, dp, dp]
        L.orc_force_stage.restype = C.c_int
        L.orc_force_stage.argtypes = [P, C.c_int64, dp, dp, dp, dp]
        L.orc_run.restype = C.c_int
        L.orc_run.argtypes = [P, dp, C.c_int64, C.c_int64]
        L.orc_macro.restype = C.c_int
        L.orc_macro.argtypes = [P, dp, C.c_int64, dp, dp, dp, dp, dp, dp]
        L.orc_set_threads.restype = None
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_get_threads.restype = C.c_int
        L.orc_get_threads.argtypes = []
        L.orc_set_threads(1)
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def set_threads(n):
    """Threads the C oracle shares its loops among (1 by default); returns the
    number it will use.  Results do not depend on it."""
    lib().orc_set_threads(int(n))
    return lib().orc_get_threads()


def cs_p0(rho, T, a=1.0, b=4.0, R=1.0):
    """Carnahan-Starling pressure, Eq. 20 (scalar)."""
    return lib().orc_cs_p0(rho, T, a, b, R)


def eos_p0(kind, rho, T, a, b, R, alpha):
    """The C oracle's p0 of EOS `kind` (a name of EOS_KIND)."""
    return lib().orc_p0(EOS_KIND[kind], rho, T, a, b, R, alpha)


def eos_mu0(kind, rho, T, a, b, R, alpha):
    return lib().orc_mu0(EOS_KIND[kind], rho, T, a, b, R, alpha)


def mrt_matrices():
    """(M, M^-1) of the C oracle's MRT collision, 9 x 9 arrays."""
    m, mi = np.zeros((9, 9)), np.zeros((9, 9))
    lib().orc_mrt_matrices(_ptr(m), _ptr(mi))
    return m, mi


def cs_mu0(rho, T, a=1.0, b=4.0, R=1.0):
    """Carnahan-Starling chemical potential without the gradient term, Eq. 21."""
    return lib().orc_cs_mu0(rho, T, a, b, R)


def cfd_alpha(order):
    """alpha of the compact scheme (Eq. 38): 1/4 gives 4th order (b = 0), 1/3 gives
    the 6th-order scheme of Eq. 39."""
    if order == 4:
        return 0.25
    if order == 6:
        return 1.0 / 3.0
    raise ValueError("compact FD order must be 4 or 6")


def cfd_line(u, alpha, h=1.0):
    """Periodic compact first derivative of the 1-D array u (Eqs. 37-38)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    d = np.empty_like(u)
    if lib().orc_cfd_line(_ptr(u), 1, _ptr(d), 1, u.size, alpha, h):
        raise ValueError("line too short")
    return d


def forcing_terms(rho, ux, uy, Fx, Fy):
    """Exact-difference forcing terms F_i of Eq. 5 at one node."""
    out = np.empty(9)
    lib().orc_forcing_terms(rho, ux, uy, Fx, Fy, _ptr(out))
    return out


class OracleSim:
    """One periodic D2Q9 simulation advanced by the C oracle, FP64."""

    def __init__(self, nx, ny, T, kappa, tau, k, fd_order, mu_max=math.inf,
                 mu_cap_steps=0, a=1.0, b=4.0, R=1.0, eos=None, mrt=None, walls_y=False,
                 wall_ux=(0.0, 0.0)):
        """`eos`: an oracle.eos.Eos (its kind, a, b, R and alpha(T) replace the
        Carnahan-Starling defaults).  `mrt`: None for BGK (Eq. 1), else the rates
        (s_e, s_eps, s_q) of the MRT collision (Eq. 4), with s_v = 1/tau and the
        conserved moments' rates 0.  `walls_y`: solid walls below the first and
        above the last row (halfway bounce-back, fields extended evenly about
        the walls for the y derivatives); `wall_ux`: the x-velocities of the
        bottom and the top wall (Ladd's moving-wall bounce-back)."""
        kind, al = 0, 1.0
        if eos is not None:
            kind, a, b, R, al = EOS_KIND[eos.kind], eos.a, eos.b, eos.R, eos.alpha(T)
        self.p = OrcParams(nx, ny, T, a, b, R, kappa, tau, k, cfd_alpha(fd_order),
                           mu_max, mu_cap_steps, kind, al)
        self.p.walls_y = 1 if walls_y else 0
        self.p.wall_ux[0], self.p.wall_ux[1] = wall_ux
        if mrt is not None:
            se, seps, sq = mrt
            sv = 1.0 / tau
            self.p.mrt = 1
            for i, v in enumerate((0.0, se, seps, 0.0, sq, 0.0, sq, sv, sv)):
                self.p.s[i] = v
        self.nx, self.ny = nx, ny
        self.t = 0
        self.f = np.zeros((9, ny, nx))

    def set_fields(self, rho, ux=None, uy=None):
        """f = f^eq(rho, u) (u = 0 where not given); time level reset to 0."""
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(self.ny, self.nx)
        ux = None if ux is None else np.ascontiguousarray(ux, np.float64).reshape(rho.shape)
        uy = None if uy is None else np.ascontiguousarray(uy, np.float64).reshape(rho.shape)
        lib().orc_feq_field(C.byref(self.p), _ptr(rho), _ptr(ux), _ptr(uy), _ptr(self.f))
        self.t = 0

    def set_populations(self, f, t=0):
        self.f[...] = f
        self.t = t

    def step(self, n):
        if lib().orc_run(C.byref(self.p), _ptr(self.f), self.t, n):
            raise RuntimeError("oracle step failed")
        self.t += n

    def fields(self):
        """(rho, vx, vy, mu_hat, Fx, Fy) of the current state."""
        shape = (self.ny, self.nx)
        rho, vx, vy, mu, Fx, Fy = (np.empty(shape) for _ in range(6))
        if lib().orc_macro(C.byref(self.p), _ptr(self.f), self.t, _ptr(rho), _ptr(vx),
                           _ptr(vy), _ptr(mu), _ptr(Fx), _ptr(Fy)):
            raise RuntimeError("oracle macro failed")
        return rho, vx, vy, mu, Fx, Fy

    def cfd_field(self, u, axis):
        """Compact derivative of a field along an axis (0: x, 1: y), or its second
        derivative along y (axis 2) as the force stage takes it, with this run's
        boundaries."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        d = np.empty_like(u)
        if lib().orc_cfd_field(C.byref(self.p), axis, _ptr(u), _ptr(d)):
            raise RuntimeError("oracle cfd failed")
        return d

    def force_stage(self, rho, t=None):
        """(mu_hat, Fx, Fy) computed from a given density field."""
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        mu, Fx, Fy = (np.empty_like(rho) for _ in range(3))
        if lib().orc_force_stage(C.byref(self.p), self.t if t is None else t, _ptr(rho),
                                 _ptr(mu), _ptr(Fx), _ptr(Fy)):
            raise RuntimeError("oracle force stage failed")
        return mu, Fx, Fy
