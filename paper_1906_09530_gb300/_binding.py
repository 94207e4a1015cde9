"""ctypes binding of libcplbm.so (include/cplbm.h): argument marshalling only.

Every function named lbm_* here calls the C function of the same name.  Device
memory and streams come from PyTorch (torch tensors' data_ptr() and
torch.cuda streams); host arrays are numpy float64.  There is no fallback: if
the library is not built, or the call fails, an exception is raised.
"""
import ctypes as C
import math
import os

import numpy as np

from . import _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_ENOTIMPL = range(7)
LBM_EOS_CS, LBM_EOS_VDW, LBM_EOS_RK, LBM_EOS_RKS, LBM_EOS_PR = range(5)
LBM_PREC_FP64, LBM_PREC_MIXED, LBM_PREC_MIXED_DF = 0, 1, 2
_PRECISIONS = {"fp64": LBM_PREC_FP64, "mixed": LBM_PREC_MIXED, "mixed_df": LBM_PREC_MIXED_DF}


class LbmGrid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("periodic_x", C.c_int32),
                ("periodic_y", C.c_int32)]


class LbmEos(C.Structure):
    _fields_ = [("kind", C.c_int32), ("a", C.c_double), ("b", C.c_double),
                ("R", C.c_double), ("omega", C.c_double)]


class LbmOpts(C.Structure):
    _fields_ = [("prec", C.c_int32), ("fd_order", C.c_int32), ("mu_max", C.c_double),
                ("mu_cap_steps", C.c_int64), ("collision", C.c_int32), ("s_e", C.c_double),
                ("s_eps", C.c_double), ("s_q", C.c_double)]


LBM_COLLIDE_BGK, LBM_COLLIDE_MRT = 0, 1
# MRT rates s_e, s_eps, s_q of Sec. 2 (after Eq. 4); s_v = 1/tau
PAPER_MRT = (1.64, 1.54, 1.9)


def _opts(prec, fd_order, mu_max, mu_cap_steps, collision, mrt_rates):
    if collision not in ("bgk", "mrt"):
        raise ValueError(collision)
    o = LbmOpts(prec, fd_order, mu_max, mu_cap_steps)
    if collision == "mrt":
        o.collision = LBM_COLLIDE_MRT
        o.s_e, o.s_eps, o.s_q = mrt_rates
    return o


class LbmInstance(C.Structure):
    _fields_ = [("grid", LbmGrid), ("T_r", C.c_double), ("kappa", C.c_double),
                ("tau", C.c_double), ("mesh_coeff", C.c_double), ("mu_max", C.c_double),
                ("mu_cap_steps", C.c_int64)]


class LbmError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {lbm_strerror(status)} (status {status})")


_lib = None
_vp, _dp, _i32, _i64 = C.c_void_p, C.POINTER(C.c_double), C.c_int32, C.c_int64


def lib():
    """The loaded library; raises ImportError if it has not been built."""
    global _lib
    if _lib is None:
        path = _build.lib_path()
        if not os.path.exists(path):
            raise ImportError(
                f"{path} is missing: build it with `python -m paper_1906_09530_gb300._build` "
                "(there is no CPU fallback)")
        L = C.CDLL(path)
        sigs = {
            "lbm_workspace_bytes": (C.c_size_t, [C.POINTER(LbmGrid), C.POINTER(LbmOpts)]),
            "lbm_init": (C.c_int, [C.POINTER(_vp), C.POINTER(LbmGrid), C.POINTER(LbmEos),
                                   C.c_double, C.c_double, C.c_double, C.c_double,
                                   C.POINTER(LbmOpts), _vp, C.c_size_t, _vp]),
            "lbm_set_fields": (C.c_int, [_vp, _vp, _vp, _vp]),
            "lbm_set_fields_device": (C.c_int, [_vp, _vp, _vp, _vp]),
            "lbm_step": (C.c_int, [_vp, _i64]),
            "lbm_step_async": (C.c_int, [_vp, _i64]),
            "lbm_check": (C.c_int, [_vp]),
            "lbm_step_timed": (C.c_int, [_vp, C.POINTER(C.c_float)]),
            "lbm_fields": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
            "lbm_fields_device": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
            "lbm_get_populations": (C.c_int, [_vp, _vp, C.POINTER(C.c_int64)]),
            "lbm_set_populations": (C.c_int, [_vp, _vp, _i64]),
            "lbm_diag": (C.c_int, [_vp, _dp, _dp, _dp, _dp]),
            "lbm_diag_noalloc": (C.c_int, [_vp, _dp, _dp, _dp, _dp]),
            "lbm_critical": (C.c_int, [C.POINTER(LbmEos), _dp, _dp]),
            "lbm_maxwell": (C.c_int, [C.POINTER(LbmEos), C.c_double, _dp, _dp]),
            "lbm_cfd": (C.c_int, [_vp, _vp, _vp, _i32, _i32, _i32, _i32, _vp]),
            "lbm_cfd_df": (C.c_int, [_vp, _vp, _vp, _vp, _i32, _i32, _i32, _i32, _vp]),
            "lbm_time": (C.c_int64, [_vp]),
            "lbm_path_flags": (C.c_int32, [_vp]),
            "lbm_set_collide_form": (C.c_int, [_vp, _i32]),
            "lbm_set_launch_mode": (C.c_int, [_vp, _i32, _i32, _i32]),
            "lbm_failed_step": (C.c_int64, [_vp]),
            "lbm_set_timeout": (C.c_int, [_vp, C.c_double]),
            "lbm_set_wall_velocity": (C.c_int, [_vp, C.c_double, C.c_double]),
            "lbm_batch_workspace_bytes": (C.c_size_t, [C.POINTER(LbmInstance), _i32,
                                                        C.POINTER(LbmOpts)]),
            "lbm_batch_init": (C.c_int, [C.POINTER(_vp), C.POINTER(LbmInstance), _i32,
                                         C.POINTER(LbmEos), C.POINTER(LbmOpts), _vp,
                                         C.c_size_t, _vp]),
            "lbm_batch_set_fields": (C.c_int, [_vp, _i32, _vp, _vp, _vp]),
            "lbm_batch_step": (C.c_int, [_vp, _i64]),
            "lbm_batch_step_timed": (C.c_int, [_vp, C.POINTER(C.c_float)]),
            "lbm_batch_fields": (C.c_int, [_vp, _i32, _vp, _vp, _vp, _vp]),
            "lbm_batch_diag": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
            "lbm_batch_autotune": (C.c_int, [_vp, _i32]),
            "lbm_batch_tile_rows": (_i32, [_vp, _i32]),
            "lbm_batch_lines_per_block": (_i32, [_vp]),
            "lbm_batch_set_lines_per_block": (C.c_int, [_vp, _i32]),
            "lbm_batch_time": (C.c_int64, [_vp, _i32]),
            "lbm_batch_failed": (C.c_int, [_vp, C.POINTER(_i32), C.POINTER(C.c_int64)]),
            "lbm_batch_set_timeout": (C.c_int, [_vp, C.c_double]),
            "lbm_batch_free": (None, [_vp]),
            "lbm_mlp_param_count": (C.c_int64, []),
            "lbm_mlp_workspace_bytes": (C.c_size_t, [_i32]),
            "lbm_mlp_init": (C.c_int, [C.POINTER(_vp), _i32, _vp, C.c_size_t, _vp]),
            "lbm_mlp_set_params": (C.c_int, [_vp, _vp]),
            "lbm_mlp_get_params": (C.c_int, [_vp, _vp]),
            "lbm_mlp_forward": (C.c_int, [_vp, _vp, _i32, _vp]),
            "lbm_mlp_loss_grad": (C.c_int, [_vp, _vp, _vp, _i32, _dp, _vp]),
            "lbm_mlp_train_step": (C.c_int, [_vp, _vp, _vp, _i32, C.c_float, _dp]),
            "lbm_mlp_set_tcgen05": (C.c_int, [_vp, _i32]),
            "lbm_mlp_tcgen05": (_i32, [_vp]),
            "lbm_mlp_free": (None, [_vp]),
            "lbm_strerror": (C.c_char_p, [C.c_int]),
            "lbm_free": (None, [_vp]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def lbm_strerror(status):
    return lib().lbm_strerror(status).decode()


def _check(status, what):
    if status != LBM_OK:
        raise LbmError(status, what)


def cs_eos(a=1.0, b=4.0, R=1.0):
    """Carnahan-Starling EOS parameters (Eq. 20; the paper's values by default)."""
    return LbmEos(LBM_EOS_CS, a, b, R, 0.0)


# EOS kinds and the paper's a, b for each (Sec. 3.2)
EOS_KINDS = {"cs": (LBM_EOS_CS, 1.0, 4.0), "vdw": (LBM_EOS_VDW, 9 / 49, 2 / 21),
             "rk": (LBM_EOS_RK, 2 / 49, 2 / 21), "rks": (LBM_EOS_RKS, 2 / 49, 2 / 21),
             "pr": (LBM_EOS_PR, 2 / 49, 2 / 21)}


def make_eos(kind="cs", a=None, b=None, R=1.0, omega=0.0):
    """EOS parameters by name ("cs", "vdw", "rk", "rks", "pr"); a and b default to
    the paper's values, omega is the acentric factor of RKS and PR."""
    k, a0, b0 = EOS_KINDS[kind]
    return LbmEos(k, a0 if a is None else a, b0 if b is None else b, R, omega)


def lbm_critical(eos=None):
    """(T_c, rho_c) of the EOS, solved on the host by the library."""
    tc, rc = C.c_double(), C.c_double()
    _check(lib().lbm_critical(C.byref(eos or cs_eos()), C.byref(tc), C.byref(rc)),
           "lbm_critical")
    return tc.value, rc.value


def lbm_maxwell(T_r, eos=None):
    """Maxwell coexistence densities (rho_g, rho_l) at T_r, solved by the library."""
    g, l = C.c_double(), C.c_double()
    _check(lib().lbm_maxwell(C.byref(eos or cs_eos()), T_r, C.byref(g), C.byref(l)),
           "lbm_maxwell")
    return g.value, l.value


def lbm_workspace_bytes(nx, ny, precision=LBM_PREC_FP64, fd_order=6):
    g = LbmGrid(nx, ny, 1, 1)
    o = LbmOpts(precision, fd_order, math.inf, 0)
    return lib().lbm_workspace_bytes(C.byref(g), C.byref(o))


def _dptr(t):
    """Device pointer of a torch tensor (must be CUDA, float64, contiguous)."""
    if t is None:
        return None
    import torch
    assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
    return t.data_ptr()


def _hptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data


def lbm_cfd(u, axis, fd_order, second=False, stream=None):
    """Compact-FD derivative(s) of a CUDA float64 tensor [ny][nx] along axis 0 (x)
    or 1 (y): returns D u, and D(D u) if `second` (Eqs. 37-39)."""
    import torch
    ny, nx = u.shape
    d1 = torch.empty_like(u)
    d2 = torch.empty_like(u) if second else None
    s = stream if stream is not None else torch.cuda.current_stream(u.device)
    _check(lib().lbm_cfd(_dptr(u), _dptr(d1), _dptr(d2), nx, ny, axis, fd_order,
                         s.cuda_stream), "lbm_cfd")
    return (d1, d2) if second else d1


def lbm_cfd_df(u_hi, u_lo, axis, fd_order, second=False, stream=None):
    """The mixed path's line solve on a double-float field given as two CUDA
    float32 tensors (hi, lo): D u in double-float rounded to float32, and D(D u)
    in float32 if `second`."""
    import torch
    ny, nx = u_hi.shape
    for t in (u_hi, u_lo):
        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
    d1 = torch.empty_like(u_hi)
    d2 = torch.empty_like(u_hi) if second else None
    s = stream if stream is not None else torch.cuda.current_stream(u_hi.device)
    _check(lib().lbm_cfd_df(u_hi.data_ptr(), u_lo.data_ptr(), d1.data_ptr(),
                            None if d2 is None else d2.data_ptr(), nx, ny, axis, fd_order,
                            s.cuda_stream), "lbm_cfd_df")
    return (d1, d2) if second else d1


class Simulation:
    """One D2Q9 run of the method (periodic, or with walls in y) on the current CUDA device.

    Owns a torch uint8 workspace and the library context.  Host inputs/outputs are
    numpy float64 [ny][nx]; device variants take/return torch float64 tensors.
    """

    def __init__(self, nx, ny, T_r, kappa, tau, mesh_coeff, fd_order=6,
                 precision="fp64", mu_max=math.inf, mu_cap_steps=0, eos=None,
                 device=None, stream=None, collision="bgk", mrt_rates=PAPER_MRT,
                 walls_y=False, wall_ux=(0.0, 0.0)):
        """`walls_y`: solid walls below the first and above the last row (else
        periodic in y); `wall_ux`: their x-velocities (bottom, top)."""
        if not walls_y and any(wall_ux):
            raise ValueError("wall_ux needs walls_y: a periodic grid has no walls to move")
        import torch
        self.nx, self.ny = nx, ny
        self.device = torch.device(device if device is not None else "cuda")
        prec = _PRECISIONS[precision]
        self.grid = LbmGrid(nx, ny, 1, 0 if walls_y else 1)
        self.opts = _opts(prec, fd_order, mu_max, mu_cap_steps, collision, mrt_rates)
        self.eos = eos or cs_eos()
        nbytes = lib().lbm_workspace_bytes(C.byref(self.grid), C.byref(self.opts))
        if nbytes == 0:
            raise LbmError(LBM_EINVAL, "lbm_workspace_bytes")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream()
            self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.ctx = C.c_void_p()
            _check(lib().lbm_init(C.byref(self.ctx), C.byref(self.grid), C.byref(self.eos),
                                  T_r, kappa, tau, mesh_coeff, C.byref(self.opts),
                                  self.ws.data_ptr(), nbytes, self.stream.cuda_stream),
                   "lbm_init")
        if walls_y and any(wall_ux):
            self.set_wall_velocity(*wall_ux)

    # -- state ------------------------------------------------------------
    def set_fields(self, rho, ux=None, uy=None):
        """Initial state from host numpy arrays (f = f^eq, Eq. 2)."""
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64)
                for a in (rho, ux, uy)]
        for a in arrs:
            if a is not None and a.size != self.nx * self.ny:
                raise ValueError("field size does not match the grid")
        _check(lib().lbm_set_fields(self.ctx, *[_hptr(a) for a in arrs]), "lbm_set_fields")

    def set_fields_device(self, rho, ux=None, uy=None):
        _check(lib().lbm_set_fields_device(self.ctx, _dptr(rho), _dptr(ux), _dptr(uy)),
               "lbm_set_fields_device")

    def step(self, n=1):
        _check(lib().lbm_step(self.ctx, n), "lbm_step")

    def step_async(self, n=1):
        _check(lib().lbm_step_async(self.ctx, n), "lbm_step_async")

    def step_timed(self):
        """One step with per-pass CUDA-event timing; returns 5 durations in ms."""
        ms = (C.c_float * 5)()
        _check(lib().lbm_step_timed(self.ctx, ms), "lbm_step_timed")
        return list(ms)

    def check(self):
        _check(lib().lbm_check(self.ctx), "lbm_check")

    @property
    def t(self):
        return lib().lbm_time(self.ctx)

    @property
    def path_flags(self):
        """Bit set: LBM_PATH_RHO_DF (2) for double-float density lines, LBM_PATH_CS_RING
        (4) for the row-ring collide-stream kernel; 0 for FP64."""
        return lib().lbm_path_flags(self.ctx)

    def set_launch_mode(self, single_graph, pdl_direct, pdl_graphs):
        """Lone steps from a one-step graph or direct launches, and programmatic
        dependent launch for direct and graph-captured passes (lbm_set_launch_mode)."""
        _check(lib().lbm_set_launch_mode(self.ctx, int(bool(single_graph)), int(bool(pdl_direct)),
                                         int(bool(pdl_graphs))), "lbm_set_launch_mode")

    def set_collide_form(self, ring_rows):
        """Mixed collide-stream form: -1 sliding window, 0 by grid size (the
        default: the row ring from 2^23 nodes), > 0 row ring with that many rows
        a block (lbm_set_collide_form)."""
        _check(lib().lbm_set_collide_form(self.ctx, int(ring_rows)), "lbm_set_collide_form")

    @property
    def failed_step(self):
        return lib().lbm_failed_step(self.ctx)

    def fields(self):
        """(rho, vx, vy, mu_hat) as host numpy arrays; v = u + F/(2 rho)."""
        out = [np.empty((self.ny, self.nx)) for _ in range(4)]
        _check(lib().lbm_fields(self.ctx, *[_hptr(a) for a in out]), "lbm_fields")
        return tuple(out)

    def fields_device(self):
        import torch
        out = [torch.empty((self.ny, self.nx), dtype=torch.float64, device=self.device)
               for _ in range(4)]
        _check(lib().lbm_fields_device(self.ctx, *[_dptr(a) for a in out]),
               "lbm_fields_device")
        return tuple(out)

    def get_populations(self):
        f = np.empty((9, self.ny, self.nx))
        t = C.c_int64()
        _check(lib().lbm_get_populations(self.ctx, _hptr(f), C.byref(t)),
               "lbm_get_populations")
        return f, t.value

    def set_populations(self, f, t=0):
        f = np.ascontiguousarray(f, dtype=np.float64)
        _check(lib().lbm_set_populations(self.ctx, _hptr(f), t), "lbm_set_populations")

    def diag(self):
        """(mass, max|v|, rho_min, rho_max), FP64 device reductions."""
        v = [C.c_double() for _ in range(4)]
        _check(lib().lbm_diag(self.ctx, *[C.byref(x) for x in v]), "lbm_diag")
        return tuple(x.value for x in v)

    def set_wall_velocity(self, u_bottom, u_top):
        _check(lib().lbm_set_wall_velocity(self.ctx, u_bottom, u_top), "lbm_set_wall_velocity")

    def set_timeout(self, seconds):
        _check(lib().lbm_set_timeout(self.ctx, seconds), "lbm_set_timeout")

    def close(self):
        if getattr(self, "ctx", None):
            lib().lbm_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent periodic instances of the mixed path advanced together
    (lbm_batch_* of the C ABI): one launch per pass for the whole batch.

    `instances` is a sequence of dicts with keys nx, ny, T_r, and optionally
    kappa (0.1), tau (1.0), k (0.5), mu_max (inf), mu_cap_steps (0); other keys
    (a caller's own bookkeeping) are ignored, except that walls are refused:
    batches are periodic only.  `precision` is "mixed" or "mixed_df", as for
    Simulation.
    """

    def __init__(self, instances, fd_order=6, precision="mixed", eos=None, device=None,
                 stream=None, collision="bgk", mrt_rates=PAPER_MRT):
        import torch
        self.n = len(instances)
        arr = (LbmInstance * self.n)()
        self.shapes = []
        for i, d in enumerate(instances):
            if d.get("walls_y") or any(d.get("wall_ux", ())):
                raise ValueError(f"instance {i}: batches are periodic only (no walls)")
            arr[i] = LbmInstance(LbmGrid(d["nx"], d["ny"], 1, 1), d["T_r"],
                                 d.get("kappa", 0.1), d.get("tau", 1.0), d.get("k", 0.5),
                                 d.get("mu_max", math.inf), d.get("mu_cap_steps", 0))
            self.shapes.append((d["ny"], d["nx"]))
        self._inst = arr
        self.opts = _opts(_PRECISIONS[precision], fd_order, math.inf, 0, collision, mrt_rates)
        self.eos = eos or cs_eos()
        nbytes = lib().lbm_batch_workspace_bytes(arr, self.n, C.byref(self.opts))
        if nbytes == 0:
            raise LbmError(LBM_EINVAL, "lbm_batch_workspace_bytes")
        self.device = torch.device(device if device is not None else "cuda")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream()
            self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.ctx = C.c_void_p()
            _check(lib().lbm_batch_init(C.byref(self.ctx), arr, self.n, C.byref(self.eos),
                                        C.byref(self.opts), self.ws.data_ptr(), nbytes,
                                        self.stream.cuda_stream), "lbm_batch_init")

    def set_fields(self, i, rho, ux=None, uy=None):
        ny, nx = self.shapes[i]
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64)
                for a in (rho, ux, uy)]
        for a in arrs:
            if a is not None and a.size != nx * ny:
                raise ValueError("field size does not match instance grid")
        _check(lib().lbm_batch_set_fields(self.ctx, i, *[_hptr(a) for a in arrs]),
               "lbm_batch_set_fields")

    def step(self, n=1):
        _check(lib().lbm_batch_step(self.ctx, n), "lbm_batch_step")

    def step_timed(self):
        """One step of the whole batch; returns the 4 pass times in ms."""
        ms = (C.c_float * 4)()
        _check(lib().lbm_batch_step_timed(self.ctx, ms), "lbm_batch_step_timed")
        return list(ms)

    def fields(self, i):
        ny, nx = self.shapes[i]
        out = [np.empty((ny, nx)) for _ in range(4)]
        _check(lib().lbm_batch_fields(self.ctx, i, *[_hptr(a) for a in out]),
               "lbm_batch_fields")
        return tuple(out)

    def diag(self):
        """Arrays (mass, max|v|, rho_min, rho_max), one entry per instance."""
        out = [np.empty(self.n) for _ in range(4)]
        _check(lib().lbm_batch_diag(self.ctx, *[_hptr(a) for a in out]), "lbm_batch_diag")
        return tuple(out)

    def autotune(self, reps=5):
        _check(lib().lbm_batch_autotune(self.ctx, reps), "lbm_batch_autotune")

    def tile_rows(self, i):
        return lib().lbm_batch_tile_rows(self.ctx, i)

    def lines_per_block(self):
        return lib().lbm_batch_lines_per_block(self.ctx)

    def set_lines_per_block(self, nl):
        _check(lib().lbm_batch_set_lines_per_block(self.ctx, nl), "lbm_batch_set_lines_per_block")

    def time(self, i):
        return lib().lbm_batch_time(self.ctx, i)

    def failed(self):
        i, t = _i32(), C.c_int64()
        _check(lib().lbm_batch_failed(self.ctx, C.byref(i), C.byref(t)), "lbm_batch_failed")
        return i.value, t.value

    def set_timeout(self, seconds):
        _check(lib().lbm_batch_set_timeout(self.ctx, seconds), "lbm_batch_set_timeout")

    def close(self):
        if getattr(self, "ctx", None):
            lib().lbm_batch_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mlp:
    """The surrogate network (lbm_mlp_* of the C ABI).  Inputs and targets are
    CUDA float32 tensors [batch][4] and [batch][256]; parameters are numpy
    float32 vectors in the library's order."""

    def __init__(self, max_batch, device=None, stream=None):
        import torch
        self.max_batch = max_batch
        self.n_params = lib().lbm_mlp_param_count()
        nbytes = lib().lbm_mlp_workspace_bytes(max_batch)
        if nbytes == 0:
            raise LbmError(LBM_EINVAL, "lbm_mlp_workspace_bytes")
        self.device = torch.device(device if device is not None else "cuda")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream()
            self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.ctx = C.c_void_p()
            _check(lib().lbm_mlp_init(C.byref(self.ctx), max_batch, self.ws.data_ptr(), nbytes,
                                      self.stream.cuda_stream), "lbm_mlp_init")

    @staticmethod
    def _f32(t, cols):
        import torch
        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
        assert t.dim() == 2 and t.shape[1] == cols
        return t.data_ptr()

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        _check(lib().lbm_mlp_set_params(self.ctx, p.ctypes.data), "lbm_mlp_set_params")

    def get_params(self):
        p = np.empty(self.n_params, dtype=np.float32)
        _check(lib().lbm_mlp_get_params(self.ctx, p.ctypes.data), "lbm_mlp_get_params")
        return p

    def forward(self, x):
        import torch
        y = torch.empty((x.shape[0], 256), dtype=torch.float32, device=x.device)
        _check(lib().lbm_mlp_forward(self.ctx, self._f32(x, 4), x.shape[0], y.data_ptr()),
               "lbm_mlp_forward")
        return y

    def loss_grad(self, x, t):
        import torch
        g = torch.empty(self.n_params, dtype=torch.float32, device=x.device)
        loss = C.c_double()
        _check(lib().lbm_mlp_loss_grad(self.ctx, self._f32(x, 4), self._f32(t, 256), x.shape[0],
                                       C.byref(loss), g.data_ptr()), "lbm_mlp_loss_grad")
        return loss.value, g

    def train_step(self, x, t, lr, want_loss=False):
        loss = C.c_double()
        _check(lib().lbm_mlp_train_step(self.ctx, self._f32(x, 4), self._f32(t, 256), x.shape[0],
                                        lr, C.byref(loss) if want_loss else None),
               "lbm_mlp_train_step")
        return loss.value if want_loss else None

    @property
    def tcgen05(self):
        """True while the forward and input-gradient products run on tcgen05."""
        return lib().lbm_mlp_tcgen05(self.ctx) == 1

    @tcgen05.setter
    def tcgen05(self, on):
        _check(lib().lbm_mlp_set_tcgen05(self.ctx, 1 if on else 0), "lbm_mlp_set_tcgen05")

    def close(self):
        if getattr(self, "ctx", None):
            lib().lbm_mlp_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
