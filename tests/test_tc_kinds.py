"""Which tcgen05.mma kinds the toolkit accepts for GB300 (sm_103a): kind::f16
(the split products' bf16 digits with fp32 accumulators) assembles, kind::i8
(int8 digits with int32 accumulators, the other exact splitting named for the
precision mode) is rejected by ptxas for this target, which is why the split
products use bf16 digits."""
import os
import shutil
import subprocess
import tempfile

import pytest

SRC = r"""
#include <stdint.h>
__global__ void k(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::KIND [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(1u) : "memory");
}
"""


def assemble(kind):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "k.cu")
    with open(src, "w") as f:
        f.write(SRC.replace("KIND", kind))
    return subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-c", src, "-o",
                           os.path.join(d, "k.o")], capture_output=True, text=True)


def test_kind_f16_assembles_for_sm_103a():
    r = assemble("f16")
    assert r.returncode == 0, r.stderr


def test_kind_i8_is_not_available_on_sm_103a():
    r = assemble("i8")
    assert r.returncode != 0 and "not supported" in r.stderr, r.stderr
