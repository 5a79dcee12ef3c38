"""Double-float arithmetic (csrc/dfloat.cuh) on the host: every operation against exact rational
(or 60-digit decimal) arithmetic on seeded random operands. The kernels that emulate FP64-class
sums on the FP32 pipe rely on these error bounds (~2^-44 relative per operation)."""
import decimal
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1811_10270_gb300", "csrc")


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("df") / "dfloat_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I" + CSRC,
                    os.path.join(HERE, "native", "dfloat_check.cpp"), "-o", exe], check=True)

    def go(pairs):
        inp = "\n".join("%.17g %.17g" % (a, b) for a, b in pairs) + "\n"
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
        return [list(map(float, l.split())) for l in out.strip().splitlines()]
    return go


def df_value(x):
    """The double-float representation of a double: hi = fl32(x), lo = fl32(x - hi) (exact)."""
    h = np.float32(x)
    l = np.float32(x - float(h))
    return Fraction(float(h)) + Fraction(float(l))


def rel(a, exact):
    exact = Fraction(exact)
    return abs(Fraction(a) - exact) / abs(exact) if exact != 0 else abs(Fraction(a))


def test_double_float_operations_are_accurate_to_about_2_pow_minus_44(run):
    rng = np.random.default_rng(7)
    n = 400
    a = rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 3, n)
    b = rng.standard_normal(n) * 10.0 ** rng.uniform(-3, 3, n)
    res = run(list(zip(a, b)))
    decimal.getcontext().prec = 60
    bound = 2.0 ** -44
    acc = Fraction(0)
    sum_abs = Fraction(0)
    for (x, y), r in zip(zip(a, b), res):
        X, Y = df_value(x), df_value(y)
        assert rel(r[0], X + Y) < bound * (abs(X) + abs(Y)) / abs(X + Y)
        assert rel(r[1], X * Y) < bound
        assert rel(r[2], X * X) < bound
        xx = Decimal_sqrt(X * X)
        assert rel(r[3], 1 / xx) < 4 * bound
        assert rel(r[4], xx) < 4 * bound
        assert rel(r[5], X / Y) < 2 * bound
        acc += X * Y
        sum_abs += abs(X * Y)
        # a long sum: error relative to the sum of magnitudes, as for an FP64 dot product
        assert abs(Fraction(r[6]) - acc) < 4 * bound * sum_abs


def Decimal_sqrt(q: Fraction) -> Fraction:
    d = decimal.Decimal(q.numerator) / decimal.Decimal(q.denominator)
    return Fraction(d.sqrt())


def test_two_sum_and_two_prod_are_error_free(run):
    # x + y and x * y with operands exactly representable in FP32: the results must be exact
    rng = np.random.default_rng(8)
    a = rng.standard_normal(200).astype(np.float32).astype(np.float64)
    b = (rng.standard_normal(200) * 1e-3).astype(np.float32).astype(np.float64)
    res = run(list(zip(a, b)))
    for (x, y), r in zip(zip(a, b), res):
        assert Fraction(r[0]) == Fraction(x) + Fraction(y)
        assert Fraction(r[1]) == Fraction(x) * Fraction(y)
