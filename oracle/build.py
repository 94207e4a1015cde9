"""Compile the C oracle (cplbm_oracle.c) into a shared library with gcc.

TEST INFRASTRUCTURE ONLY: the oracle is the independent FP64 CPU restatement of
the method that the tests compare the CUDA library against.  Building it is not
using it; only the tests, the smoke check and the benchmark's CPU-baseline leg
load the result.

Flags: -O2 without fast-math, and -ffp-contract=off so that no multiply-add is
fused on either x86 or Arm hosts (the oracle's bits do not depend on the host);
-fopenmp where gcc supports it (the thread count is 1 unless the caller sets it
with orc_set_threads).
"""
import os
import platform
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cplbm_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")


def lib_path() -> str:
    return os.path.join(OUT_DIR, f"liboracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    out = lib_path()
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(SRC)):
        return out
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wextra", "-o", tmp, SRC, "-lm"]
    # with OpenMP when the compiler has it (the loops over lines and nodes are
    # shared among threads; results do not depend on the thread count)
    r = subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True))
