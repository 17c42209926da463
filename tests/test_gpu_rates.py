"""Measured throughput of the GB300 pipes the multiple-double path can use
(tests/harness/rates.cu): FP64 DFMA/DADD instructions, FP32 FFMA, INT32 IMAD,
the warp-level matrix instructions mma.sync for bf16, int8 and f64, and
tcgen05.mma kind::f16 (M = 128, operands in shared memory in the split
products' layout) at N = 16 ... 256.
These rates set the roofline denominators of the md kernels (FP64
instructions per second) and decide which pipe the split products use.
Run with -s to see the numbers."""
import ctypes as C
import os
import shutil
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NAMES = ["FP64 DFMA instr/s", "FP64 DADD instr/s", "FP32 FFMA instr/s", "INT32 IMAD instr/s",
         "HMMA bf16 m16n8k16 flop/s", "IMMA s8 m16n8k32 op/s", "DMMA f64 m8n8k4 flop/s"]


def test_pipe_rates():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = os.path.join(tempfile.mkdtemp(), "librates.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared", "-Xcompiler",
                    "-fPIC", "-o", out, os.path.join(ROOT, "tests", "harness", "rates.cu")], check=True)
    L = C.CDLL(out)
    L.probe_rates.argtypes = [C.POINTER(C.c_double), C.c_int]
    r = (C.c_double * 7)()
    assert L.probe_rates(r, 7) == 0
    for name, v in zip(NAMES, r):
        print(f"{name:28s} {v / 1e12:10.3f} T")
    assert all(v > 0 for v in r)
    # the FP64 issue rate the md rooflines use: 2 instructions/clk/SM x 152 SMs
    # x 2.07 GHz = 0.629 T/s; a probe far from it would make those fractions wrong
    assert 0.3e12 < r[0] < 0.8e12
    L.probe_tcgen05.argtypes = [C.POINTER(C.c_double), C.c_int]
    t = (C.c_double * 4)()
    assert L.probe_tcgen05(t, 4) == 0
    for n, cyc in zip((16, 64, 128, 256), t):
        print(f"tcgen05.mma kind::f16 M=128 N={n:3d}: {cyc:7.1f} cycles, {128 * n * 16 / cyc:7.0f} MAC/clk/SM")
    # 128 x 256 x 16 at the nominal bf16 rate (about 4096 MAC/clk/SM) is 128 cycles
    assert 100 < t[3] < 400 and t[0] <= t[3]
