"""The exact-to-FP64 rounding of the FP64 tensor-core and integer-limb kernels,
compiled for the host, against exact rational rounding; and the integer-limb
stencil's limb split and 729-tap row sums (wrapped middle word) against exact
integers.

The seven-digit mode product (STFD_FP64TC7) and the integer-limb band products
(STFD_OP_FX64) form each result as an exact integer and round it once, to
nearest even, with integer instructions (fp64_round.cuh, shared by host and
device). These cases check that claim bit for bit against Python's correctly
rounded Fraction -> float conversion: random accumulators of up to nine
27-bit-limb products, exact cancellations, pairs of products at scales up to
2^16 apart, the seven-digit recombination of FP32-exact partial sums, and scales
that push results into the subnormal range and past the largest finite value.
"""
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1909_07309_gb300", "csrc")


def _cuda_include():
    for base in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if base and os.path.exists(os.path.join(base, "include", "cuda_runtime.h")):
            return os.path.join(base, "include")
    return None


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx, inc = shutil.which("g++"), _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("rnd") / "rounding_driver")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", inc, "-I", CSRC, os.path.join(HERE, "rounding_driver.cpp"),
                    "-o", exe], check=True, capture_output=True)
    return exe


def _raw(exe, lines):
    return subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                          check=True).stdout.splitlines()


def _run(exe, lines):
    return [struct.unpack("<d", struct.pack("<Q", int(v)))[0] for v in _raw(exe, lines)]


def _ref(fr):
    try:
        return float(fr)   # correctly rounded (ties to even), subnormals included
    except OverflowError:
        return float("inf") if fr > 0 else float("-inf")


def _same(a, b):
    return struct.pack("<d", a) == struct.pack("<d", b) or (a == 0.0 and b == 0.0)


def _acc(rng):
    """A band-product accumulator: up to 9 taps of C, U with |C|, |U| < 2^53
    split into 27-bit limbs (high signed, low in [0, 2^27))."""
    hh = mm = ll = 0
    for _ in range(rng.randint(1, 9)):
        bits = rng.choice([53, 53, 40, 27, 8, 2])
        C = rng.randint(-(2 ** bits - 1), 2 ** bits - 1)
        U = rng.choice([rng.randint(-(2 ** 53 - 1), 2 ** 53 - 1), 0, 1, -1, 2 ** 52, -(2 ** 52)])
        ch, cl, uh, ul = C >> 27, C & (2 ** 27 - 1), U >> 27, U & (2 ** 27 - 1)
        hh += ch * uh
        ll += cl * ul
        mm += (ch + cl) * (uh + ul)
    return hh, mm, ll


def _value(a):
    hh, mm, ll = a
    return hh * 2 ** 54 + (mm - hh - ll) * 2 ** 27 + ll


SCALES = [2150, 2100, 2200, 1050, 1000, 980, 960, 3100, 3200]   # normal, subnormal, overflow


def test_single_products_round_exactly(driver):
    rng = random.Random(11)
    cases = [(_acc(rng), rng.choice(SCALES)) for _ in range(20000)]
    got = _run(driver, ["acc %d %d %d %d" % (a[0], a[1], a[2], se) for a, se in cases])
    for (a, se), g in zip(cases, got):
        assert _same(g, _ref(Fraction(_value(a)) * Fraction(2) ** (se - 2150))), (a, se, g)


def test_product_pairs_sum_exactly_then_round(driver):
    rng = random.Random(12)
    cases = []
    for _ in range(15000):
        x = _acc(rng)
        y = tuple(-v for v in x) if rng.random() < 0.05 else _acc(rng)   # exact cancellation too
        sx = rng.choice(SCALES)
        cases.append((x, sx, y, sx - rng.randint(-16, 16)))
    got = _run(driver, ["pair %d %d %d %d %d %d %d %d" % (x[0], x[1], x[2], sx, y[0], y[1], y[2], sy)
                        for x, sx, y, sy in cases])
    for (x, sx, y, sy), g in zip(cases, got):
        exact = Fraction(_value(x)) * Fraction(2) ** (sx - 2150) + Fraction(_value(y)) * Fraction(2) ** (sy - 2150)
        assert _same(g, _ref(exact)), (x, sx, y, sy, g)


def test_seven_digit_recombination_rounds_exactly(driver):
    rng = random.Random(13)
    cases = []
    for _ in range(20000):
        lim = rng.choice([2 ** 23, 2 ** 20, 2 ** 12, 200, 2])
        I = [rng.randint(-lim + 1, lim - 1) for _ in range(7)]
        if rng.random() < 0.05:
            I = [0] * rng.randint(1, 6) + [rng.randint(-9, 9) for _ in range(7)]
            I = I[-7:]
        cases.append((I, rng.choice([0, -20, 60, -1000, -1060, -1080, -1100, -1130, 960, 990])))
    got = _run(driver, ["c7 " + " ".join(map(str, I)) + " %d" % se for I, se in cases])
    for (I, se), g in zip(cases, got):
        Z = sum(I[c] * 256 ** (6 - c) for c in range(7))
        assert _same(g, _ref(Fraction(Z) * Fraction(2) ** se)), (I, se, g)


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _round_half_away(fr):
    n = abs(fr.numerator) * 2 + fr.denominator
    q = n // (2 * fr.denominator)
    return q if fr >= 0 else -q


def test_stencil_balanced_limbs_of_fp64_entries(driver):
    """U = round(m 2^{max(e,1) - E}), halves away from zero, split as
    h 2^27 + l with l in [-2^26, 2^26): the entry's value in units of
    2^{E - 1075}."""
    rng = random.Random(14)
    cases = []
    for _ in range(20000):
        x = rng.choice([rng.uniform(-1, 1), rng.gauss(0, 1) * 2.0 ** rng.randint(-40, 40), 5e-324 * rng.randint(1, 9),
                        2.0 ** rng.randint(-1074, 1023) * rng.choice([1, -1, 1.5])])
        e = max(1, (_bits(x) >> 52) & 0x7FF)
        cases.append((x, min(2046, e + rng.choice([0, 0, 1, 2, 20, 52, 53, 54, 60, 70]))))
    out = _raw(driver, ["bl %d %d" % (_bits(x), E) for x, E in cases])
    for (x, E), line in zip(cases, out):
        h, l = map(int, line.split())
        assert -(2 ** 26) <= l < 2 ** 26 and abs(h) <= 2 ** 26, (x, E, h, l)
        assert h * 2 ** 27 + l == _round_half_away(Fraction(x) / Fraction(2) ** (E - 1075)), (x, E, h, l)


# Largest |h + l| of a balanced split, 2^27 - 2: the middle word's terms reach
# 2^54 and 729 of them pass 2^63 (the accumulation wraps).
WRAP = (2 ** 26 - 1) * 2 ** 27 + 2 ** 26 - 1


def _row(rng, n, worst=False):
    lim = 2 ** 53 - 1
    if worst:   # every product at its largest, one sign: the sums' bounds are reached
        s = rng.choice([1, -1])
        return [(s * rng.choice([WRAP, lim]), WRAP) for _ in range(n)]
    return [(rng.randint(-lim, lim) >> rng.choice([0, 0, 0, 20, 45]), rng.randint(-lim, lim) >> rng.choice([0, 0, 30]))
            for _ in range(n)]


def _exact(row):
    return sum(c * u for c, u in row)


def _split(v):
    lo = ((v + 2 ** 26) % 2 ** 27) - 2 ** 26
    return (v - lo) >> 27, lo


def test_stencil_worst_rows_wrap_the_middle_word():
    """The worst-case rows used below do overflow a signed 64-bit middle sum."""
    (h, l) = _split(WRAP)
    assert 729 * (h + l) ** 2 >= 2 ** 63 and abs(h) <= 2 ** 26 and -(2 ** 26) <= l < 2 ** 26


def test_stencil_row_sums_of_729_taps_round_exactly(driver):
    rng = random.Random(15)
    cases = []
    for k in range(600):
        n = rng.choice([729, 729, 125, 27, 1])
        cases.append((_row(rng, n, worst=k % 50 == 0), rng.choice([2150, 2100, 2200, 1040, 3000])))
    lines = ["stw %d %d " % (se, len(r)) + " ".join("%d %d" % cu for cu in r) for r, se in cases]
    for (r, se), g in zip(cases, _run(driver, lines)):
        assert _same(g, _ref(Fraction(_exact(r)) * Fraction(2) ** (se - 2150))), (se, g)


def test_stencil_row_pairs_within_2_pow_10_sum_exactly(driver):
    rng = random.Random(16)
    cases = []
    for k in range(400):
        x = _row(rng, 729, worst=k % 40 == 0)
        y = [(-c, u) for c, u in x] if k % 17 == 0 else _row(rng, rng.choice([729, 343]), worst=k % 40 == 1)
        sx = rng.choice([2150, 2120, 1050])
        cases.append((x, sx, y, sx + rng.randint(-10, 10)))
    lines = ["stp %d %d %s %d %d %s" % (sx, len(x), " ".join("%d %d" % cu for cu in x), sy, len(y),
                                        " ".join("%d %d" % cu for cu in y)) for x, sx, y, sy in cases]
    for (x, sx, y, sy), g in zip(cases, _run(driver, lines)):
        exact = Fraction(_exact(x)) * Fraction(2) ** (sx - 2150) + Fraction(_exact(y)) * Fraction(2) ** (sy - 2150)
        assert _same(g, _ref(exact)), (sx, sy, g)
