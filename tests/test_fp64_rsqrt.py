"""Host check of the Cholesky pivots' 1/sqrt(d) and sqrt(d) (one third-order
step from a single-precision seed, exponent split and format moves by integer
operations): within 2 ulps of the exact values over the whole normal range,
also from seeds up to 16 float ulps off (the device seed is the hardware
approximation, within 2 ulps, of the truncated operand, not the correctly
rounded float), and
the library functions for zero, subnormal, negative and non-finite pivots."""
from __future__ import annotations

import math
import os
import random
import shutil
import struct
import subprocess
from decimal import Decimal, getcontext

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1710_08471_gb300", "csrc")
getcontext().prec = 60


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("rsqrt") / "rsqrt_check")
    # -ffp-contract=off: fma() is the only fused operation, as in the kernel
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC,
                    os.path.join(HERE, "native", "rsqrt_check.cpp"), "-o", exe], check=True)

    def go(lines):
        out = subprocess.run([exe], input="".join(lines), capture_output=True, text=True, check=True).stdout
        return [[struct.unpack("<d", int(w, 16).to_bytes(8, "little"))[0] for w in ln.split()]
                for ln in out.strip().split("\n")]

    return go


def _bits(x):
    return struct.unpack("<q", struct.pack("<d", x))[0]


def _ulps(got, exact: Decimal):
    u = math.ulp(float(exact))
    return abs(Decimal(got) - exact) / Decimal(u)


def test_pivot_rsqrt_and_sqrt(run):
    rng = random.Random(5)
    ds = [2.0 ** rng.uniform(-1020, 1020) for _ in range(4000)]
    ds += [1.0, 2.0, 4.0, 3.999999999999999, 1.0000000000000002, 2.0 ** -1022, 2.0 ** 1023 * 1.9999999999999998,
           0.25, 1e-300, 1e300]
    got = run([f"0 {_bits(d)} 0\n" for d in ds])
    worst_r = worst_l = 0
    for d, (r, l) in zip(ds, got):
        s = Decimal(d).sqrt()
        worst_r = max(worst_r, _ulps(r, 1 / s))
        worst_l = max(worst_l, _ulps(l, s))
    assert worst_r <= 2 and worst_l <= 2, (worst_r, worst_l)


def test_newton_from_perturbed_seeds(run):
    rng = random.Random(6)
    fs = [rng.uniform(1.0, 4.0) for _ in range(2000)] + [1.0, 3.9999999999999996]
    lines = [f"1 {_bits(f)} {p}\n" for f in fs for p in (-16, -8, -3, 0, 3, 8, 16)]
    got = run(lines)
    for (f, p), (y,) in zip([(f, p) for f in fs for p in (-16, -8, -3, 0, 3, 8, 16)], got):
        assert _ulps(y, 1 / Decimal(f).sqrt()) <= 2, (f, p, y)


def test_non_normal_pivots_take_the_library(run):
    ds = [0.0, -1.0, 5e-324, 2.0 ** -1070, float("inf"), float("nan")]
    got = run([f"0 {_bits(d)} 0\n" for d in ds])
    for d, (r, l) in zip(ds, got):
        want_l = math.sqrt(d) if d >= 0 or math.isnan(d) else float("nan")
        if math.isnan(want_l):
            assert math.isnan(l)
        else:
            assert l == want_l
