"""Which tcgen05.mma operand kinds the sm_103a target accepts (CPU only).

The split-precision path could cut FP64 entries into INT8 digits multiplied
with exact INT32 accumulation (tcgen05.mma kind::i8) instead of BF16 digits
with FP32 group sums (kind::f16). This checks, with the toolkit's own
assembler, that kind::i8 is not an instruction of sm_103a (GB300), while the
kind::f16 form the library uses is; so no INT8 split-precision variant is
built.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import tempfile

import pytest

KERNEL = r"""
#include <cstdint>
__global__ void k(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::KIND [%0], %1, %2, %3, p;\n}\n"
               ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
"""


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


def _compile(kind: str) -> subprocess.CompletedProcess:
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "k.cu")
        with open(src, "w") as f:
            f.write(KERNEL.replace("KIND", kind))
        return subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-cubin", "-o",
                               os.path.join(d, "k.cubin"), src], capture_output=True, text=True, timeout=300)


def test_kind_f16_is_an_sm103a_instruction():
    r = _compile("f16")
    assert r.returncode == 0, r.stderr


def test_kind_i8_is_not_an_sm103a_instruction():
    r = _compile("i8")
    assert r.returncode != 0
    assert "kind::i8" in r.stderr and "sm_103a" in r.stderr, r.stderr
