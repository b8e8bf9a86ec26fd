"""Host check of the split-precision integer arithmetic: the slicing of FP64
entries into balanced base-256 digits, and the accumulator -> FP64
conversion.

The kernel turns its two int64 fixed-point accumulators into a double with
integer operations: exactly (hi 2^32 + lo, or X 2^24 + Y) for the Gram, and
to within one ulp for the Q-form. The same routines, compiled for the host,
are compared with exact rational arithmetic (Python's Fraction -> float rounds
to nearest, ties to even) on random, tie, carry, sign and subnormal cases.
"""
from __future__ import annotations

import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1710_08471_gb300", "csrc")


@pytest.fixture(scope="module")
def conv(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("conv") / "fixed_conv_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "native", "fixed_conv_check.cpp"),
                    "-o", exe], check=True)

    def run(cases, mode=0):
        inp = "".join(f"{mode} {h} {l} {e}\n" for h, l, e in cases)
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split()
        return [struct.unpack("<d", int(w, 16).to_bytes(8, "little"))[0] for w in out]

    return run


def exact(h, l, e, shift=32):
    v = Fraction(h * (1 << shift) + l) * (Fraction(2) ** e)
    try:
        return float(v)
    except OverflowError:
        return float("inf") if v > 0 else float("-inf")


def _check(conv, cases):
    got = conv(cases)
    for (h, l, e), g in zip(cases, got):
        want = exact(h, l, e)
        assert struct.pack("<d", g) == struct.pack("<d", want), (h, l, e, g, want)


def test_random(conv):
    rng = random.Random(7)
    cases = []
    for _ in range(20000):
        bh, bl = rng.randint(0, 61), rng.randint(0, 61)
        h = rng.randint(-(1 << bh), 1 << bh)
        l = rng.randint(-(1 << bl), 1 << bl)
        cases.append((h, l, rng.randint(-120, 40)))
    _check(conv, cases)


def test_ties_carries_and_signs(conv):
    cases = []
    for k in range(0, 40):
        # exactly half an ulp above a representable value (ties to even both ways)
        for m in ((1 << 53) - 1, (1 << 53) - 2, (1 << 52) + 1, (1 << 52)):
            t = (2 * m + 1) << k
            for sgn in (1, -1):
                v = sgn * t
                cases.append((v >> 32, v - ((v >> 32) << 32), -10))
                cases.append(((v >> 32) - 1, v - ((v >> 32) << 32) + (1 << 32), 3))
    # rounding carry into the exponent, zero, hi/lo cancellation, lo < 0
    cases += [(0, 0, 0), (1, -(1 << 32), 5), (0, (1 << 54) - 1, 0), ((1 << 21) - 1, (1 << 32) - 1, 0),
              (-(1 << 40), 123, -7), (5, -(1 << 61), 2), (-(1 << 61), -(1 << 61), -200)]
    _check(conv, cases)


def test_subnormal_and_overflow(conv):
    rng = random.Random(3)
    cases = [(rng.randint(-(1 << 40), 1 << 40), rng.randint(-(1 << 50), 1 << 50), rng.randint(-1200, -1050))
             for _ in range(3000)]
    cases += [(1, 0, -1106), (0, 1, -1074), (0, 1, -1075), (0, 3, -1076), (0, 2, -1076), ((1 << 40), 0, 980),
              (-(1 << 40), 0, 990)]
    _check(conv, cases)


def _ulp(x):
    import math

    return math.ulp(x)


def test_xy_exact(conv):
    rng = random.Random(11)
    cases = [(rng.randint(-(1 << 60), 1 << 60) >> rng.randint(0, 60), rng.randint(-(1 << 54), 1 << 54) >> rng.randint(0, 54),
              rng.randint(-150, 30)) for _ in range(20000)]
    cases += [(0, 0, 0), (-1, (1 << 24) - 1, 0), (1, -(1 << 24), 3), (-(1 << 60), -(1 << 54), -100), (255, -1, -1080)]
    got = conv(cases, 1)
    for (x, y, e), g in zip(cases, got):
        want = exact(x, y, e, 24)
        assert struct.pack("<d", g) == struct.pack("<d", want), (x, y, e, g, want)


def test_xy_fast_within_one_ulp(conv):
    rng = random.Random(12)
    cases = [(rng.randint(-(1 << 60), 1 << 60) >> rng.randint(0, 60), rng.randint(-(1 << 54), 1 << 54) >> rng.randint(0, 54),
             rng.randint(-150, 30)) for _ in range(30000)]
    # X alone near the shift threshold, Y cancelling X, zero
    for b in range(30, 45):
        cases += [((1 << b) - 1, -(1 << 53), -60), (-(1 << b), (1 << 54) - 1, -60), (1 << b, -(1 << (b + 24)) // (1 << 24), 0)]
    cases += [(0, 0, 0), (0, 5, -3), (-7, 0, 2), (1, -(1 << 24), 0)]
    got = conv(cases, 2)
    for (x, y, e), g in zip(cases, got):
        t = x * (1 << 24) + y
        want = exact(x, y, e, 24)
        if abs(x) < (1 << 38):  # no bits dropped: correctly rounded
            assert struct.pack("<d", g) == struct.pack("<d", want), (x, y, e, g, want)
        else:
            assert abs(Fraction(g) - Fraction(t) * Fraction(2) ** e) <= Fraction(_ulp(want)), (x, y, e, g, want)


# ---------------------------------------------------------------- slicing

@pytest.fixture(scope="module")
def slicer(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("slice") / "fixed_conv_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "native", "fixed_conv_check.cpp"),
                    "-o", exe], check=True)

    def run(cases):
        lines = []
        for x, e, S in cases:
            bits = struct.unpack("<q", struct.pack("<d", x))[0]
            lines.append(f"3 {bits} {S} {e}\n")
        out = subprocess.run([exe], input="".join(lines), capture_output=True, text=True, check=True).stdout
        res = []
        for ln in out.strip().split("\n"):
            w = [int(t) for t in ln.split()]
            res.append((w[0], w[1:]))
        return res

    return run


def _peel(v, S):
    """Balanced base-256 digits by the definition: the signed low byte, then
    (v - d) / 256, repeated; the rest is the top digit."""
    d = [0] * S
    for s in range(S - 1, 0, -1):
        lo = v & 0xFF
        lo = lo - 256 if lo >= 128 else lo
        d[s] = lo
        v = (v - lo) >> 8
    d[0] = v
    return d


def test_slicing_digits(slicer):
    """Every entry x with |x| < 2^e becomes v = x 2^(7 + 8(S-1) - e) rounded
    to an integer (half away from zero, error <= 1/2, exact when no bits are
    dropped), and S balanced digits with v = sum d_s 256^(S-1-s), d_s in
    [-128, 127] below the top digit, equal to the digits peeled off one byte
    at a time."""
    rng = random.Random(11)
    cases = []
    for _ in range(6000):
        S = rng.choice((6, 7))
        e = rng.randint(-60, 60)
        kind = rng.random()
        if kind < 0.6:
            x = rng.uniform(-1.0, 1.0) * 2.0 ** e
        elif kind < 0.8:
            x = rng.uniform(-1.0, 1.0) * 2.0 ** (e - rng.randint(1, 80))
        else:  # just below 2^e, and ties in the last kept place
            k = 7 + 8 * (S - 1) - e
            x = (rng.choice((1, -1)) * ((1 << (7 + 8 * (S - 1))) - rng.randint(0, 3)) + rng.choice((0, 0.5))) * 2.0 ** -k
            if abs(x) >= 2.0 ** e:
                x = 0.0
        cases.append((x, e, S))
    cases += [(0.0, 0, 7), (-0.0, 3, 6), (5e-324, -1021, 7), (-2.0 ** -1030, -1025, 6)]
    got = slicer(cases)
    for (x, e, S), (v, d) in zip(cases, got):
        k = 7 + 8 * (S - 1) - e
        t = Fraction(x) * Fraction(2) ** k
        assert abs(t) < Fraction(2) ** (7 + 8 * (S - 1)) or x == 0.0
        assert abs(Fraction(v) - t) <= Fraction(1, 2), (x, e, S, v)
        if t.denominator == 1:
            assert v == t, (x, e, S, v)
        assert sum(di * 256 ** (S - 1 - i) for i, di in enumerate(d)) == v
        assert all(-128 <= di <= 127 for di in d[1:]) and abs(d[0]) <= 128
        assert d == _peel(v, S), (x, e, S)
