"""The general double-float kernel terms (csrc/pair_df.cuh: the FP64-class all-pairs sums of close drop
pairs, the near-field sums and the all-pairs form without quantised positions) on the host, against
exact arithmetic (rationals, 60-digit decimals) on seeded random geometry.

Each operand is split as the library stages it (FP32 value plus FP32 remainder, about 48 bits); the
reference takes the staged values exactly, so what is measured is the terms' arithmetic. The coordinate
difference is formed in double-float from two offsets of size ~1, so a pair r apart keeps ~2^-47 / r of
relative accuracy in the difference; every term is within 2^-44 (1 + 1/r) of its scale: |s|/r (single
layer), |s|/r^2 (double layer: the dot product with the normal may cancel), |f|/r (Stokeslet) and
|u||n|/r^2 (stresslet).
"""
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
    exe = str(tmp_path_factory.mktemp("dft") / "df_term_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I" + CSRC,
                    os.path.join(HERE, "native", "df_term_check.cpp"), "-o", exe], check=True)

    def go(rows):
        inp = "".join("%d %s\n" % (k, " ".join("%.17g" % v for v in vals)) for k, vals in rows)
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
        return [list(map(float, l.split())) for l in out.strip().splitlines()]
    return go


def staged(v):
    """The exact value of the library's (FP32 value, FP32 remainder) split of a double."""
    h = np.float32(v)
    l = np.float32(v - float(h))
    return Fraction(float(h)) + Fraction(float(l))


def _unit(rng):
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


def cases(rng, n):
    """Source node on a drop of radius U(0.8, 1.3) about 0, target r away in a random direction (r
    log-uniform in [0.01, 10]); densities N(0,1) times a random scale, unit normals."""
    out = []
    for _ in range(n):
        V = _unit(rng) * rng.uniform(0.8, 1.3)
        r = 10.0 ** rng.uniform(-2, 1)
        T = V + _unit(rng) * r
        f = rng.standard_normal(3) * 10.0 ** rng.uniform(-2, 2)
        u = rng.standard_normal(3) * 10.0 ** rng.uniform(-2, 2)
        out.append(list(T) + list(V) + list(f) + list(u) + list(_unit(rng)) + list(_unit(rng)))
    return out


def D(x):
    return decimal.Decimal(x.numerator) / decimal.Decimal(x.denominator)


def exact(kind, vals):
    """The accumulators' exact values and the scale each is measured against."""
    decimal.getcontext().prec = 60
    T, V, f, u, n, N = (vals[3 * k:3 * k + 3] for k in range(6))
    d = [staged(T[k]) - staged(V[k]) for k in range(3)]
    f = [staged(x) for x in f]
    u = [staged(x) for x in u]
    n = [staged(x) for x in n]
    N = [staged(x) for x in N]
    r2 = sum(x * x for x in d)
    ri = 1 / D(r2).sqrt()
    r = float(1 / ri)
    dot = lambda a, b: sum(a[k] * b[k] for k in range(3))
    fn = float(np.linalg.norm([float(x) for x in f]))
    if kind == 1:
        return [D(f[0]) * ri], abs(float(f[0])) / r
    if kind == 0:
        return [D(f[0]) * D(dot(d, N)) * ri ** 3], abs(float(f[0])) / r ** 2
    un = float(np.linalg.norm([float(x) for x in u])) * float(np.linalg.norm([float(x) for x in n]))
    hu, hn, hf = D(dot(d, u)), D(dot(d, n)), D(dot(d, f))
    out = []
    for k in range(3):
        t = decimal.Decimal(0)
        if kind in (2, 3):
            t += D(f[k]) * ri + D(d[k]) * hf * ri ** 3
        if kind in (2, 4):
            t += D(d[k]) * hu * hn * ri ** 5
        out.append(t)
    scale = {2: fn / r + un / r ** 2, 3: fn / r, 4: un / r ** 2}[kind]
    return out, scale


@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4])
def test_terms_against_exact_arithmetic(run, kind):
    rng = np.random.default_rng(10 + kind)
    rows = [(kind, v) for v in cases(rng, 300)]
    if kind in (0, 1):
        rows = [(kind, v[:6] + [v[6], 0.0, 0.0] + v[9:]) for _, v in rows]
    got = run(rows)
    worst = 0.0
    for (k, vals), g in zip(rows, got):
        ref, scale = exact(k, vals)
        T, V = np.array(vals[0:3]), np.array(vals[3:6])
        r = float(np.linalg.norm(T - V))
        for a, b in zip(g, ref):
            err = float(abs(decimal.Decimal(a) - b)) / scale
            worst = max(worst, err / (1.0 + 1.0 / r))
    assert worst < 2.0 ** -44, worst
