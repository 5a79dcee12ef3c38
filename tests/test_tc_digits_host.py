"""The digit arithmetic behind the tensor-core kernels with FP64-class accuracy (csrc/tc_digits.cuh)
on the host, against exact rational arithmetic: digit bounds (every digit exact in bfloat16 and every
diagonal sum of a K-step product exact in FP32), the reconstruction of each split value, the
recombination of the six diagonal sums, and a whole digit-split product with the shape of the
row analysis' Fourier stage (Section 2.1) against the exact dot products."""
import math
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1811_10270_gb300", "csrc")


@pytest.fixture(scope="module")
def tcd(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("tcd") / "tc_digits_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I" + CSRC,
                    os.path.join(HERE, "native", "tc_digits_check.cpp"), "-o", exe], check=True)

    def go(lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                             check=True).stdout
        return out.strip().splitlines()
    return go


def f32(x):
    return float(np.float32(x))


def split_df(x):
    """double-float (hi, lo) of a double: hi = fl32(x), lo = fl32(x - hi)"""
    h = f32(x)
    return h, f32(x - h)


def digits6(tcd, pairs):
    out = tcd(["D %s %s" % (float(h).hex(), float(l).hex()) for h, l in pairs])
    return [list(map(int, s.split())) for s in out]


def test_digits_of_double_float_values(tcd):
    rng = np.random.default_rng(11)
    mags = 2.0 ** rng.uniform(-30, 7, 4000)
    xs = rng.choice([-1.0, 1.0], 4000) * mags * rng.uniform(0.5, 1.0, 4000)
    pairs = [split_df(x) for x in xs]
    pairs = [(h, l) for h, l in pairs if abs(h) < 128.0]
    for (h, l), d in zip(pairs, digits6(tcd, pairs)):
        assert abs(d[5]) <= 128 and abs(d[4]) <= 64 and abs(d[3]) <= 64
        assert abs(d[2]) <= 72 and abs(d[1]) <= 65 and abs(d[0]) <= 65
        val = sum(Fraction(d[j]) * Fraction(2) ** (7 * (j - 5)) for j in range(6))
        assert abs(val - (Fraction(h) + Fraction(l))) <= Fraction(1, 2 ** 35)


def test_digits_of_table_values(tcd):
    rng = np.random.default_rng(12)
    xs = rng.uniform(-1.0, 1.0, 2000) * 2.0 ** rng.integers(-12, 1, 2000)
    out = tcd(["H %s %d" % (float(x).hex(), 1) for x in xs])
    for x, s in zip(xs, out):
        d = list(map(int, s.split()))
        assert all(abs(v) <= 64 for v in d[:5]) and abs(d[5]) <= 128
        assert sum(d[j] * 128 ** j for j in range(6)) == round(Fraction(x) * 2 ** 41)


def test_combine_of_six_diagonal_sums(tcd):
    rng = np.random.default_rng(13)
    rows = []
    for _ in range(2000):
        a = [int(v) for v in rng.integers(-(2 ** 24) + 1, 2 ** 24, 6)]
        a[0] = int(rng.integers(2 ** 18, 2 ** 24)) * int(rng.choice([-1, 1]))   # a dominant top sum
        rows.append(a)
    out = tcd(["C " + " ".join(float(v).hex() for v in a) for a in rows])
    for a, s in zip(rows, out):
        hi, lo = (float.fromhex(t) for t in s.split())
        exact = sum(Fraction(a[i]) * Fraction(2) ** (-7 * i) for i in range(6))
        # the top three terms join exactly (two-sums); the three lowest, weights 2^-21 and below, are
        # one FP32 sum below 2^4 in magnitude, so they carry at most half an FP32 unit there, 2^-20
        assert abs(Fraction(hi) + Fraction(lo) - exact) <= Fraction(1, 2 ** 20) + abs(exact) * Fraction(1, 2 ** 44)


def test_digit_split_product_matches_exact_dot_products(tcd):
    """Rows of 132 double-float values times the 132 x 66 cos/sin table of the degree-32 Fourier stage:
    per row a power-of-two scale 2^(7-e) (max |hi| < 2^e), six digits per value, table digits at
    2^41, the 21 products with j_a + j_b >= 5 summed per diagonal (each sum an integer below 2^24, so
    FP32 accumulation is exact), recombined and scaled by 2^(e-13)."""
    rng = np.random.default_rng(14)
    K, nrow, p = 132, 6, 32
    k = np.arange(K)
    cols = [np.cos(2 * np.pi * (m * k % K) / K) for m in (0, 1, 7, p)] + \
           [np.sin(2 * np.pi * (m * k % K) / K) for m in (1, 13, p)]
    tdig = []
    for c in cols:
        tdig.append([list(map(int, s.split())) for s in tcd(["H %s 1" % float(v).hex() for v in c])])
    for r in range(nrow):
        x = rng.standard_normal(K) * 10.0 ** rng.uniform(-3, 3) * np.exp(-0.05 * k * (r % 3))
        pairs = [split_df(v) for v in x]
        e = math.frexp(max(abs(h) for h, _ in pairs))[1]
        sc = 2.0 ** (7 - e)
        adig = digits6(tcd, [(f32(h * sc), f32(l * sc)) for h, l in pairs])
        for c, td in zip(cols, tdig):
            acc = [0] * 6
            for kk in range(K):
                for ja in range(6):
                    for jb in range(5 - ja, 6):
                        acc[ja + jb - 5] += adig[kk][ja] * td[kk][jb]
            assert all(abs(a) < 2 ** 24 for a in acc)
            hi, lo = (float.fromhex(t) for t in tcd(["C " + " ".join(float(a).hex() for a in acc[::-1])])[0].split())
            got = (Fraction(hi) + Fraction(lo)) * Fraction(2) ** (e - 13)
            exact = sum(Fraction(h) * Fraction(float(cv)) + Fraction(l) * Fraction(float(cv)) for (h, l), cv in zip(pairs, c))
            bound = sum(abs(Fraction(h) + Fraction(l)) * abs(Fraction(float(cv))) for (h, l), cv in zip(pairs, c))
            # the neglected products (j_a + j_b < 5) and the digits' rounding stay near 2^-40 of
            # sum |x||T| (2^-40.0 at worst here); leaving out the lowest kept diagonal costs 2^-34
            assert abs(got - exact) <= Fraction(1, 2 ** 39) * bound


def _constexpr(src, name):
    import re
    txt = open(os.path.join(CSRC, src)).read()
    return int(re.search(r"constexpr int %s = (\d+);" % name, txt).group(1))


def test_diagonal_sums_stay_exact_at_the_largest_k():
    """Worst case of every diagonal sum from the digit bounds (row digits d5..d0 up to 128, 64, 64, 72,
    65, 65; table digits up to 128 and 64) at the longest K each tensor-core kernel accepts, read from
    the kernels' own limits: the Fourier stage runs K = 4(p+1) longitudes with 2(p+1) <= kNT, the
    rotations K <= kNmax (padded blocks), the Legendre stage K = 2p+2 <= kKmax latitudes. Below 2^24,
    FP32 accumulation in tensor memory is exact. The kernels assert the same bound at compile time
    (static_assert on diag_sums_exact); this recomputes it independently of the C++ expression."""
    a_max = {5: 128, 4: 64, 3: 64, 2: 72, 1: 65, 0: 65}
    b_max = {5: 128, 4: 64, 3: 64, 2: 64, 1: 64, 0: 64}
    ks = {"fourier": 2 * _constexpr("dft_tc.cu", "kNT"), "rotation": _constexpr("rot_tc.cu", "kNmax"),
          "legendre": _constexpr("leg_tc.cu", "kKmax")}
    assert ks["fourier"] >= 160 and ks["rotation"] >= 80 and ks["legendre"] >= 80
    for name, K in ks.items():
        for s in range(6):
            worst = K * sum(a_max[ja] * b_max[s + 5 - ja] for ja in range(6) if 0 <= s + 5 - ja <= 5)
            assert worst < 2 ** 24, (name, K, s, worst)
