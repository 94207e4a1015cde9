"""Compile-time resources of the device kernels, read from ptxas's own report
(nvcc -Xptxas -v), without a GPU.

  * no kernel of the library spills registers to local memory or keeps a stack
    frame: the launch bounds that fix each kernel's blocks per SM are met
    without spilling;
  * every collide-stream kernel of the mixed path (periodic, walled, batched)
    uses at most 48 registers, so that 10 blocks of 128 threads fit on an SM
    (48 x 128 x 10 = 61 440 of 65 536 registers), the occupancy its memory-
    level parallelism relies on.
"""
import os
import re
import subprocess
import tempfile

import pytest

from paper_1906_09530_gb300 import _build

CSRC = os.path.join(os.path.dirname(_build.__file__), "csrc")
ENTRY = re.compile(r"Compiling entry function '([^']+)'.*?(\d+) bytes stack frame, "
                   r"(\d+) bytes spill stores, (\d+) bytes spill loads\s*\n"
                   r"ptxas info\s+: Used (\d+) registers", re.S)
pytestmark = pytest.mark.slow


@pytest.fixture(scope="module")
def entries():
    try:
        nvcc = _build._nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    srcs = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    out = {}
    with tempfile.TemporaryDirectory() as d:
        procs = [(s, subprocess.Popen([nvcc] + _build.flags() + ["-Xptxas", "-v", "-c",
                                       os.path.join(CSRC, s), "-o", os.path.join(d, s + ".o")],
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT,
                                      text=True)) for s in srcs]
        for s, p in procs:
            txt, _ = p.communicate(timeout=600)
            assert p.returncode == 0, txt[-2000:]
            out[s] = [(m.group(1), int(m.group(2)), int(m.group(3)), int(m.group(4)),
                       int(m.group(5))) for m in ENTRY.finditer(txt)]
    assert sum(len(v) for v in out.values()) >= 20
    return out


def test_no_kernel_spills(entries):
    bad = [(s, name[:80], stack, st, ld) for s, es in entries.items()
           for name, stack, st, ld, _ in es if stack or st or ld]
    assert not bad, bad


def test_collide_stream_register_budget(entries):
    """The sliding-window kernels keep ten blocks of four warps an SM (48
    registers).  The row-ring kernel's occupancy is set by its 42 KB of shared
    memory (five blocks of 128 threads an SM): registers must not lower that."""
    cs = [(name, regs) for name, _, _, _, regs in entries["kernels_mixed.cu"]
          if "k_cs_mixed" in name and "ring" not in name]
    assert len(cs) >= 6  # periodic, walled and batched, each BGK and MRT
    assert all(regs <= 48 for _, regs in cs), cs
    ring = [(name, regs) for name, _, _, _, regs in entries["kernels_mixed.cu"]
            if "k_cs_mixed_ring" in name]
    assert len(ring) == 2  # BGK and MRT
    assert all(regs * 128 * 5 <= 65536 for _, regs in ring), ring
