"""The C-ABI library without a GPU: it loads, exports every symbol the header
declares, validates arguments before touching CUDA, and its host
thermodynamics agree with the oracle's (two independent solvers)."""
import ctypes as C
import math
import os
import re

import pytest

import paper_1906_09530_gb300 as P
from paper_1906_09530_gb300 import _binding as B
from oracle import thermo

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "cplbm.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = P.lib()
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_critical_point_agrees_with_oracle():
    tc, rc = P.lbm_critical()
    otc, orc = thermo.critical_point()
    assert tc == pytest.approx(otc, rel=1e-12)
    assert rc == pytest.approx(orc, rel=1e-10)
    # other a, b, R
    eos = P.cs_eos(2.0, 3.0, 1.5)
    tc2, rc2 = P.lbm_critical(eos)
    otc2, orc2 = thermo.critical_point(2.0, 3.0, 1.5)
    assert tc2 == pytest.approx(otc2, rel=1e-12) and rc2 == pytest.approx(orc2, rel=1e-10)


@pytest.mark.parametrize("T_r", [0.95, 0.7, 0.6, 0.5, 0.45, 0.35, 0.3, 0.2, 0.16])
def test_maxwell_agrees_with_oracle(T_r):
    g, l = P.lbm_maxwell(T_r)
    og, ol = thermo.maxwell(T_r)
    assert l == pytest.approx(ol, rel=1e-12)
    assert g == pytest.approx(og, rel=1e-9)


@pytest.mark.parametrize("kind", ["vdw", "rk", "rks", "pr", "cs"])
def test_other_eos_thermodynamics_agree_with_oracle(kind):
    """The library's critical point (maximum of the closed-form spinodal
    temperature, refined on B'A'' = B''A') and Maxwell pair (nested bisection)
    against the oracle's generic solver (brentq on the spinodal, bounded
    maximisation, brentq on log p_sat)."""
    from oracle import eos as E
    omega = 0.344 if kind in ("rks", "pr") else 0.0
    e = P.make_eos(kind, omega=omega)
    o = E.Eos(kind, omega=omega)
    tc, rc = P.lbm_critical(e)
    otc, orc = o.critical_point()
    assert tc == pytest.approx(otc, rel=1e-12)
    assert rc == pytest.approx(orc, rel=1e-7)
    for t_r in (0.9, 0.7, 0.5, 0.35):
        g, l = P.lbm_maxwell(t_r, e)
        og, ol = o.maxwell(t_r)
        assert l == pytest.approx(ol, rel=1e-11)
        assert g == pytest.approx(og, rel=1e-9)


def test_workspace_bytes_validation():
    assert P.lbm_workspace_bytes(1024, 1024, P.LBM_PREC_MIXED, 6) > 9 * 1024 * 1024 * 4 * 2
    assert P.lbm_workspace_bytes(1024, 1024, P.LBM_PREC_FP64, 6) > 9 * 1024 * 1024 * 8 * 2
    assert P.lbm_workspace_bytes(4, 1024, P.LBM_PREC_FP64, 6) == 0     # nx < 8
    assert P.lbm_workspace_bytes(64, 64, P.LBM_PREC_FP64, 5) == 0      # bad order
    assert P.lbm_workspace_bytes(64, 64, 7, 6) == 0                    # bad precision


def test_mrt_rates_validated():
    g = B.LbmGrid(64, 64, 1, 1)
    for rates, ok in (((1.64, 1.54, 1.9), True), ((0.0, 1.5, 1.5), False),
                      ((1.5, 2.0, 1.5), False), ((1.5, 1.5, -1.0), False)):
        o = B._opts(B.LBM_PREC_MIXED, 6, math.inf, 0, "mrt", rates)
        assert (P.lib().lbm_workspace_bytes(C.byref(g), C.byref(o)) > 0) == ok
    o = B.LbmOpts(B.LBM_PREC_MIXED, 6, math.inf, 0)
    o.collision = 7
    assert P.lib().lbm_workspace_bytes(C.byref(g), C.byref(o)) == 0


def _init(**kw):
    args = dict(nx=64, ny=64, T_r=0.6, kappa=0.1, tau=1.0, k=0.5, order=6, ws=256, wsb=1 << 40)
    args.update(kw)
    ctx = C.c_void_p()
    g = B.LbmGrid(args["nx"], args["ny"], args.get("px", 1), args.get("py", 1))
    o = B.LbmOpts(B.LBM_PREC_FP64, args["order"], math.inf, 0)
    st = P.lib().lbm_init(C.byref(ctx), C.byref(g), C.byref(P.cs_eos()), args["T_r"],
                          args["kappa"], args["tau"], args["k"], C.byref(o), args["ws"],
                          args["wsb"], None)
    return st, ctx


@pytest.mark.parametrize("bad", [dict(tau=0.5), dict(kappa=0.0), dict(k=0.0), dict(k=1.5),
                                 dict(T_r=1.0), dict(T_r=0.0), dict(nx=7), dict(order=8),
                                 dict(ws=0), dict(ws=100)])
def test_init_rejects_bad_arguments(bad):
    st, ctx = _init(**bad)
    assert st == B.LBM_EINVAL and not ctx.value


def test_init_small_workspace_and_walls():
    st, _ = _init(wsb=16)
    assert st == B.LBM_ENOMEM
    st, _ = _init(px=0)
    assert st == B.LBM_ENOTIMPL


def test_cfd_rejects_bad_arguments():
    lib = P.lib()
    assert lib.lbm_cfd(None, 256, None, 8, 8, 0, 6, None) == B.LBM_EINVAL
    assert lib.lbm_cfd(256, 512, None, 8, 8, 2, 6, None) == B.LBM_EINVAL
    assert lib.lbm_cfd(256, 512, None, 8, 8, 0, 5, None) == B.LBM_EINVAL
    assert lib.lbm_cfd(256, 256, None, 8, 8, 0, 6, None) == B.LBM_EINVAL  # aliasing


def test_strerror_and_null_ctx():
    assert "unstable" in P.lbm_strerror(B.LBM_EUNSTABLE)
    lib = P.lib()
    assert lib.lbm_step(None, 1) == B.LBM_EINVAL
    assert lib.lbm_time(None) == -1
    lib.lbm_free(None)
    assert lib.lbm_set_wall_velocity(None, 0.0, 0.0) == B.LBM_EINVAL
    assert lib.lbm_path_flags(None) == -1
    # launch and kernel choices, and the batch's and the network's
    assert lib.lbm_set_collide_form(None, 0) == B.LBM_EINVAL
    assert lib.lbm_set_launch_mode(None, 1, 1, 0) == B.LBM_EINVAL
    assert lib.lbm_batch_lines_per_block(None) == -1
    assert lib.lbm_batch_set_lines_per_block(None, 16) == B.LBM_EINVAL
    assert lib.lbm_mlp_set_tcgen05(None, 1) == B.LBM_EINVAL
    assert lib.lbm_mlp_tcgen05(None) == -1


def test_oracle_and_library_share_nothing():
    """The CUDA library and its binding never import, include or load the oracle,
    and the oracle never imports the library."""
    root = os.path.dirname(os.path.dirname(__file__))
    pkg = os.path.join(root, "paper_1906_09530_gb300")
    bad_pkg = re.compile(r"^\s*(import|from)\s+oracle\b|#include\s*[<\"].*oracle|liboracle",
                         re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                assert not bad_pkg.search(open(os.path.join(dirpath, f)).read()), f
    bad_orc = re.compile(r"paper_1906_09530_gb300|cplbm\.h|libcplbm")
    for f in os.listdir(os.path.join(root, "oracle")):
        if f.endswith((".py", ".c")):
            assert not bad_orc.search(open(os.path.join(root, "oracle", f)).read()), f


def test_batch_init_validates_before_any_device_work():
    """Batches hold periodic instances of the mixed path only; the checks run
    before the library touches a device."""
    import ctypes as C
    lib = P.lib()
    eos = P.cs_eos()

    def init(periodic_y=1, prec=B.LBM_PREC_MIXED, order=6):
        inst = (B.LbmInstance * 1)()
        inst[0] = B.LbmInstance(B.LbmGrid(64, 64, 1, periodic_y), 0.7, 0.1, 1.0, 0.5,
                                float("inf"), 0)
        opts = B.LbmOpts(prec, order, float("inf"), 0)
        out = C.c_void_p()
        return lib.lbm_batch_init(C.byref(out), inst, 1, C.byref(eos), C.byref(opts), None, 0,
                                  None), out
    st, out = init(periodic_y=0)
    assert st == B.LBM_ENOTIMPL and not out.value
    st, _ = init(prec=B.LBM_PREC_FP64)
    assert st == B.LBM_ENOTIMPL
    st, _ = init(order=5)
    assert st == B.LBM_EINVAL
    st, _ = init()  # valid instance, but no workspace
    assert st == B.LBM_EINVAL


def test_header_is_plain_c():
    """include/cplbm.h is a C header: it compiles as C99 with -pedantic."""
    import shutil
    import subprocess
    import tempfile
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(__file__))
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.c")
        with open(src, "w") as f:
            f.write('#include "cplbm.h"\nint main(void) { lbm_grid g = {8, 8, 1, 0}; '
                    '(void)g; return 0; }\n')
        r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                            os.path.join(root, "include"), "-c", src, "-o",
                            os.path.join(d, "t.o")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


C_CONSUMER = r"""
#include <math.h>
#include <stdio.h>
#include "cplbm.h"
int main(void)
{
    lbm_eos cs = {LBM_EOS_CS, 1.0, 4.0, 1.0, 0.0};
    lbm_grid grid = {1024, 1024, 1, 1}, bad = {4, 1024, 1, 1};
    lbm_opts opts = {LBM_PREC_MIXED, 6, INFINITY, 0, LBM_COLLIDE_BGK, 0.0, 0.0, 0.0};
    double tc, rc, g, l;
    if (lbm_critical(&cs, &tc, &rc) != LBM_OK || lbm_maxwell(&cs, 0.5, &g, &l) != LBM_OK)
        return 1;
    printf("%.17g %.17g %.17g %.17g %zu %zu %d\n", tc, rc, g, l,
           lbm_workspace_bytes(&grid, &opts), lbm_workspace_bytes(&bad, &opts),
           lbm_strerror(LBM_EINVAL) != NULL && lbm_strerror(LBM_EINVAL)[0] != 0);
    return 0;
}
"""


def test_plain_c_program_links_and_calls_the_host_entry_points():
    """A C99 program built against include/cplbm.h and linked to the library
    calls the host-only entry points (no GPU needed) and gets the oracle's
    thermodynamics."""
    import shutil
    import subprocess
    import tempfile
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    so = P.lib()._name
    root = os.path.dirname(os.path.dirname(__file__))
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "consumer.c"), os.path.join(d, "consumer")
        with open(src, "w") as f:
            f.write(C_CONSUMER)
        r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                            os.path.join(root, "include"), src, "-o", exe, so,
                            "-Wl,-rpath," + os.path.dirname(so), "-lm"],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
        assert r.returncode == 0, r.stderr
    tc, rc, g, l, ws, ws_bad, msg = r.stdout.split()
    otc, orc = thermo.critical_point()
    og, ol = thermo.maxwell(0.5)
    assert float(tc) == pytest.approx(otc, rel=1e-12)
    assert float(rc) == pytest.approx(orc, rel=1e-10)
    assert float(g) == pytest.approx(og, rel=1e-9) and float(l) == pytest.approx(ol, rel=1e-12)
    # mixed: two FP32 population buffers (72 B) and eight 4-byte field planes (32 B)
    assert 1024 * 1024 * 104 <= int(ws) <= 1024 * 1024 * 105
    assert int(ws_bad) == 0 and msg == "1"


_SCALAR = {"double": C.c_double, "float": C.c_float, "int32_t": C.c_int32,
           "int64_t": C.c_int64, "size_t": C.c_size_t, "lbm_status": C.c_int}


def _declarations():
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for ret, name, params in re.findall(
            r"((?:const\s+)?[A-Za-z_]\w*\s*\*?)\s*\b(lbm_\w+)\s*\(([^)]*)\)\s*;", src):
        ps = [p.strip() for p in params.replace("\n", " ").split(",")]
        out[name] = (ret.strip(), [] if ps == ["void"] else ps)
    return out


def _matches(ctype_decl, ct):
    """Whether a ctypes type `ct` passes the C type of a declaration (a
    parameter with its name, or a return type) without truncation."""
    words = ctype_decl.replace("*", " * ").split()
    if "*" in words:
        if words[:2] == ["const", "char"] and words.count("*") == 1 and len(words) <= 4:
            return ct is C.c_char_p or ct is C.c_void_p
        return ct is C.c_void_p or ct is C.c_char_p or issubclass(ct, C._Pointer)
    base = [w for w in words if w != "const"][0]
    if base == "void":
        return ct is None
    return ct is _SCALAR[base]


def test_binding_signatures_match_the_header():
    """Every function the header declares has a ctypes signature in the
    binding, with the same number of parameters, a pointer type wherever the
    header has a pointer, and the exact scalar type elsewhere (a default int
    return or argument would truncate a size_t, an int64_t or a pointer)."""
    lib = P.lib()
    decls = _declarations()
    assert len(decls) == len(declared_symbols())
    for name, (ret, params) in decls.items():
        fn = getattr(lib, name)
        assert fn.argtypes is not None, name
        assert len(fn.argtypes) == len(params), (name, params, fn.argtypes)
        assert _matches(ret, fn.restype), (name, ret, fn.restype)
        for p, ct in zip(params, fn.argtypes):
            assert _matches(p, ct), (name, p, ct)


def test_struct_layouts_match_the_header():
    """The binding's ctypes structures have the size and the field offsets that
    a C compiler gives the header's structs (so no field is read across
    padding)."""
    import shutil
    import subprocess
    import tempfile
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = {"lbm_grid": B.LbmGrid, "lbm_eos": B.LbmEos, "lbm_opts": B.LbmOpts,
               "lbm_instance": B.LbmInstance}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "cplbm.h"',
             'int main(void) {']
    for cname, py in structs.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'    printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ['    return 0;', '}']
    root = os.path.dirname(os.path.dirname(__file__))
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines) + "\n")
        r = subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I",
                            os.path.join(root, "include"), src, "-o", exe],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        out = subprocess.run([exe], capture_output=True, text=True, timeout=60).stdout
    got = {}
    for line in out.split("\n"):
        if line:
            cname, key, val = line.split()
            got[(cname, key)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)


def test_workspace_bytes_beyond_two_to_the_31_nodes():
    """A 46 341 x 46 341 grid has more than 2^31 nodes (about 233 GB of mixed
    workspace, within a GB300's memory): the size is computed without
    overflow: mixed, two FP32 population buffers and eight FP32 planes (104
    bytes per node); FP64, two FP64 population buffers and seven FP64 planes
    (200 bytes per node); plus alignment."""
    n = 46_341
    assert n * n > 2 ** 31
    g = B.LbmGrid(n, n, 1, 1)
    for prec, per_node in ((B.LBM_PREC_MIXED, 104), (B.LBM_PREC_FP64, 200)):
        o = B._opts(prec, 6, math.inf, 0, "bgk", None)
        ws = P.lib().lbm_workspace_bytes(C.byref(g), C.byref(o))
        assert ws == pytest.approx(per_node * n * n, rel=1e-6), (prec, ws)


def test_wall_velocity_without_walls_is_refused_before_any_device_work():
    with pytest.raises(ValueError, match="walls_y"):
        P.Simulation(16, 16, 0.6, 0.1, 1.0, 0.5, wall_ux=(0.05, 0.0))


def test_batch_refuses_walls_before_any_device_work():
    with pytest.raises(ValueError, match="periodic only"):
        P.Batch([dict(nx=16, ny=16, T_r=0.6), dict(nx=16, ny=16, T_r=0.6, walls_y=True)])
