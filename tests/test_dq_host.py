"""The FP64-class pair terms on quantised positions (csrc/pair_dq.cuh) on the host, against exact
arithmetic (rationals, 60-digit decimals) on seeded random geometry.

* The premise: with Q = 23 - ceil(log2 B) and offsets below B, the quantised parts of two offsets and
  their difference are exact in FP32.
* For pairs at least 2^(19-Q) apart (where the all-pairs kernel uses these terms) 1/r, the single-layer
  term s/r and the target-normal double-layer term s (d.n0)/r^3 (relative to s/r^2) are good to
  2^-42 relative, the stresslet's 1/r^5 to five times that.
* Closer pairs lose accuracy as ~2^-(Q+23)/r (the FP32 remainders below the quantum), which is why the
  kernel keeps the general double-float terms for them.
"""
import decimal
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
def run(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("dq") / "dq_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I" + CSRC,
                    os.path.join(HERE, "native", "dq_check.cpp"), "-o", exe], check=True)

    def go(rows):
        inp = "".join("%d %s\n" % (q, " ".join("%.17g" % v for v in vals)) for q, vals in rows)
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
        return [list(map(float, l.split())) for l in out.strip().splitlines()]
    return go


def _unit(rng):
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


def _cases(rng, Q, n, centre_dist):
    """n pairs: source node on a drop of radius U(0.8, 1.3) about 0, target node on a drop of the same
    size whose centre lies centre_dist() away; strength N(0,1) with a random scale, unit target normal."""
    out = []
    for _ in range(n):
        v = _unit(rng) * rng.uniform(0.8, 1.3)
        c = _unit(rng) * centre_dist()
        T = c + _unit(rng) * rng.uniform(0.8, 1.3)
        s = rng.standard_normal() * 10.0 ** rng.uniform(-2, 2)
        out.append((Q, list(T) + list(v) + [s] + list(_unit(rng))))
    return out


def _exact(vals):
    decimal.getcontext().prec = 60
    T, V, s, n0 = vals[0:3], vals[3:6], vals[6], vals[7:10]
    d = [Fraction(T[k]) - Fraction(V[k]) for k in range(3)]
    r2 = sum(x * x for x in d)
    r = decimal.Decimal(r2.numerator) / decimal.Decimal(r2.denominator)
    r = r.sqrt()
    ri = 1 / r
    dn = sum(d[k] * Fraction(n0[k]) for k in range(3))
    D = lambda f: decimal.Decimal(f.numerator) / decimal.Decimal(f.denominator)
    return (ri, r2, D(Fraction(s)) * ri, D(Fraction(s)) * D(dn) * ri * ri * ri,
            abs(s) * math.sqrt(float(r2)) * float(ri) ** 3, ri ** 5)


def _rel(x, ref):
    ref = decimal.Decimal(ref) if not isinstance(ref, decimal.Decimal) else ref
    return float(abs(decimal.Decimal(x) - ref) / abs(ref))


@pytest.mark.parametrize("Q", [19, 17])
def test_quantised_differences_are_exact(Q):
    rng = np.random.default_rng(Q)
    B = 2.0 ** (23 - Q)
    qs, qi = 2.0 ** Q, 2.0 ** -Q
    for _ in range(2000):
        a, b = rng.uniform(-B, B, 2)
        ha, hb = math.floor(a * qs + 0.5) * qi, math.floor(b * qs + 0.5) * qi
        fa, fb = np.float32(ha), np.float32(hb)
        assert float(fa) == ha and float(fb) == hb
        assert Fraction(float(np.float32(fa - fb))) == Fraction(ha) - Fraction(hb)


@pytest.mark.parametrize("Q", [19, 17])
def test_far_pairs_are_fp64_class(run, Q):
    rng = np.random.default_rng(100 + Q)
    B = 2.0 ** (23 - Q)
    # centres 2.3 .. (B - 2.7) apart: every offset and difference stays below B per component
    cases = _cases(rng, Q, 300, lambda: rng.uniform(2.3, B - 2.7))
    res = run(cases)
    far = 2.0 ** (19 - Q)
    checked = 0
    for (q, vals), (ri, r2, sl, dl, r5) in zip(cases, res):
        e_ri, e_r2, e_sl, e_dl, dl_scale, e_r5 = _exact(vals)
        if float(e_r2) < far * far:
            continue
        checked += 1
        assert _rel(ri, e_ri) < 2.0 ** -42
        assert _rel(sl, e_sl) < 2.0 ** -42
        assert abs(float(decimal.Decimal(dl) - e_dl)) < 2.0 ** -42 * dl_scale
        assert _rel(r5, e_r5) < 5 * 2.0 ** -42      # the fifth power: five times the bound on 1/r
    assert checked > 200


def test_close_pairs_lose_accuracy_with_the_quantum(run):
    """Q = 19: pairs 0.02 to 1 apart keep 1/r within 2^-(Q+21)/r (the remainders' precision, ~2^-(Q+23)
    absolute, with margin) -- looser than the far pairs' 2^-42 at the closest distances."""
    Q = 19
    rng = np.random.default_rng(7)
    cases = []
    for _ in range(300):
        v = _unit(rng) * 1.0
        T = v + _unit(rng) * rng.uniform(0.02, 1.0)
        cases.append((Q, list(T) + list(v) + [1.0] + list(_unit(rng))))
    res = run(cases)
    for (q, vals), (ri, r2, sl, dl, r5) in zip(cases, res):
        e_ri, e_r2, _, _, _, _ = _exact(vals)
        r = math.sqrt(float(e_r2))
        assert _rel(ri, e_ri) < 2.0 ** -(Q + 21) / r
