"""Pins of the interpolation step of the nearly-singular method (oracle/nearinterp.py, Section 2.1 last
paragraph) against closed forms on the unit sphere and a converged brute force on a perturbed drop.

Closed forms outside the unit sphere, |x| = r > 1, with the 1/(4 pi) of the operators:
  * single layer of a density Y_nm:  Y_nm(x/r) r^-(n+1) / (2n+1)  (the Legendre generating function
    and the addition theorem);
  * its field E = -grad:  ((n+1) Y_nm x/r - grad_S2 Y_nm) r^-(n+2) / (2n+1);
  * Stokeslet of a constant density c:  (4/3) [(3/4)(I/r + x x^T/r^3) + (1/4)(I/r^3 - 3 x x^T/r^5)] c
    (the flow past a translating sphere, whose traction is uniform; on the sphere it is (4/3) c);
  * stresslet of a constant density: 0 outside (D[c] = 2c, c, 0 inside, on, outside).
"""
import math

import numpy as np
import pytest

import inputs
from oracle import nearinterp as NI, nearsing, operators, sh

P = 6


def _unit(rng):
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)


def _angles(x):
    r = np.linalg.norm(x)
    xh = x / r
    return r, xh, xh[2], math.hypot(xh[0], xh[1]), math.atan2(xh[1], xh[0])


def exact_single_layer(n, c, x, p=P):
    r, _, ct, st, ph = _angles(x)
    S = sh.basis(p, np.array([ct]), np.array([st]), np.array([ph]))[:, 0]
    return (c @ S) * r ** (-(n + 1)) / (2 * n + 1)


def exact_field(n, c, x, p=P):
    r, xh, ct, st, ph = _angles(x)
    S, St, Sp = sh.basis(p, np.array([ct]), np.array([st]), np.array([ph]), derivs=True)
    th_hat = np.array([ct * math.cos(ph), ct * math.sin(ph), -st])
    ph_hat = np.array([-math.sin(ph), math.cos(ph), 0.0])
    Y = c @ S[:, 0]
    gY = (c @ St[:, 0]) * th_hat + (c @ Sp[:, 0]) * ph_hat
    return ((n + 1) * Y * xh - gY) * r ** (-(n + 2)) / (2 * n + 1)


def exact_stokeslet_of_constant(cv, x):
    r = np.linalg.norm(x)
    X = np.outer(x, x)
    I = np.eye(3)
    return (4.0 / 3.0) * ((0.75 * (I / r + X / r ** 3) + 0.25 * (I / r ** 3 - 3.0 * X / r ** 5)) @ cv)


@pytest.fixture(scope="module")
def sphere():
    drop = operators.DropGeom(inputs.sphere_coef(P), P, 1.0)
    lap = {}
    for n in (2, P):
        c = np.zeros(sh.ncoef(P))
        c[sh.idx(n, 1)] = 1.0
        lap[n] = (c, NI.Source(drop, "lsl", c), NI.Source(drop, "ladl", c))
    cv = np.array([0.3, -0.5, 0.8])
    C = np.zeros((3, sh.ncoef(P)))
    C[:, 0] = cv * math.sqrt(4.0 * math.pi)
    return drop, lap, cv, NI.Source(drop, "sto_s", C), NI.Source(drop, "sto_d", C)


def test_closest_point():
    """On the unit sphere x* = x0/|x0| and d = |x0| - 1; on a perturbed drop a point placed at distance d
    along the normal of a surface point comes back to that point and distance."""
    rng = np.random.default_rng(1)
    sph = operators.DropGeom(inputs.sphere_coef(P), P, 1.0)
    for _ in range(4):
        v = _unit(rng)
        x0 = v * (1.0 + rng.uniform(0.001, 0.3))
        _, _, xs, ns, d = NI.closest_point(sph, x0)
        assert np.abs(xs - v).max() < 1e-13 and np.abs(ns - v).max() < 1e-13
        assert abs(d - (np.linalg.norm(x0) - 1.0)) < 1e-13
    drop = operators.DropGeom(inputs.perturbed_coef(P, rng, 1.0, (0.0, 0.0, 0.0)), P, 1.0)
    for _ in range(4):
        _, _, xs, ns, _ = NI.closest_point(drop, _unit(rng) * 1.1)
        dd = rng.uniform(0.005, 0.2)
        th, ph, xs2, ns2, d2 = NI.closest_point(drop, xs + dd * ns)
        assert np.abs(xs2 - xs).max() < 1e-12 and abs(d2 - dd) < 1e-12
        assert np.abs(ns2 - ns).max() < 1e-11


def test_exterior_limits_on_the_sphere(sphere):
    """The limits from outside at surface points: single layer Y/(2n+1), field ((n+1) Y n - grad Y)/(2n+1),
    Stokeslet (4/3) c, stresslet 0 (the principal value c minus the jump c)."""
    drop, lap, cv, ss, sd = sphere
    rng = np.random.default_rng(2)
    for _ in range(3):
        th, ph = rng.uniform(0.1, 3.0), rng.uniform(0.0, 2 * math.pi)
        x = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        n0 = _unit(rng)
        for n, (c, sl, fl) in lap.items():
            assert abs(NI.exterior_limit(drop, "lsl", c, th, ph) - exact_single_layer(n, c, x)) < 1e-13
            assert abs(NI.exterior_limit(drop, "ladl", c, th, ph, n0=n0, phi_coef=fl.phi)
                       - exact_field(n, c, x) @ n0) < 1e-12
        assert np.abs(NI.exterior_limit(drop, "sto_s", ss.dens, th, ph) - 4.0 / 3.0 * cv).max() < 1e-12
        assert np.abs(NI.exterior_limit(drop, "sto_d", sd.dens, th, ph)).max() < 1e-12


def test_interpolation_on_the_sphere(sphere):
    """Targets at 0.02 - 1.19 h_j from the unit sphere: the method (interpolation below 1.2 h_j) is within
    2e-6 (single layer of Y_nm, n = 2 and 6), 3e-5 (its field), 1e-6 (Stokeslet) and 5e-7 (stresslet)
    of the closed forms. Closest in, the four times upsampled rule alone is off by a thousand times more."""
    drop, lap, cv, ss, sd = sphere
    rng = np.random.default_rng(3)
    h = ss.h
    for dd in (0.02, 0.1, 0.3, 0.6, 1.0, 1.19):
        for _ in range(2):
            v, n0 = _unit(rng), _unit(rng)
            x0 = v * (1.0 + dd * h)
            for n, (c, sl, fl) in lap.items():
                val, dh = NI.value(sl, x0)
                assert abs(dh - dd) < 1e-9
                assert abs(val - exact_single_layer(n, c, x0)) < 2e-6
                assert abs(NI.value(fl, x0, n0)[0] - exact_field(n, c, x0) @ n0) < 3e-5
            assert np.abs(NI.value(ss, x0)[0] - exact_stokeslet_of_constant(cv, x0)).max() < 1e-6
            assert np.abs(NI.value(sd, x0)[0]).max() < 5e-7
    x0 = _unit(rng) * (1.0 + 0.05 * h)
    c, sl, fl = lap[P]
    n0 = _unit(rng)
    assert abs(float(fl.upsampled(x0[:, None], n0)[0]) - exact_field(P, c, x0) @ n0) > \
        1e3 * abs(NI.value(fl, x0, n0)[0] - exact_field(P, c, x0) @ n0)
    assert np.abs(sd.upsampled(x0[:, None])[:, 0]).max() > 1e3 * np.abs(NI.value(sd, x0)[0]).max()


def test_interpolation_on_a_perturbed_drop_against_brute_force():
    """A perturbed drop (p = 4; on-surface rule on the degree 4p+3 grid so that the limit is converged) with
    random densities: at 0.3 and 0.45 h_j the method agrees with the regular rule on the 32 times upsampled
    grid, itself converged there (16 and 32 times agree to 1e-8), to 2e-6."""
    p = 4
    rng = np.random.default_rng(4)
    drop = operators.DropGeom(inputs.perturbed_coef(p, rng, 1.0, (0.0, 0.0, 0.0)), p, 1.0, q=4 * p + 3)
    sig = inputs.random_density(p, rng, 1).ravel()
    f3 = inputs.random_density(p, rng, 3)
    srcs = {"lsl": NI.Source(drop, "lsl", sig), "ladl": NI.Source(drop, "ladl", sig),
            "sto_s": NI.Source(drop, "sto_s", f3), "sto_d": NI.Source(drop, "sto_d", f3)}
    g16 = {k: NI._Grid(drop, s.dens, 16) for k, s in srcs.items()}
    g32 = {k: NI._Grid(drop, s.dens, 32) for k, s in srcs.items()}
    h = srcs["lsl"].h
    for dd in (0.3, 0.45):
        for _ in range(2):
            _, _, xs, ns, _ = NI.closest_point(drop, _unit(rng) * 1.2)
            x0 = xs + dd * h * ns
            n0 = _unit(rng)
            for k, s in srcs.items():
                nk = n0 if k == "ladl" else None
                val = np.atleast_1d(NI.value(s, x0, nk)[0])
                b16 = g16[k].rule(k, x0[:, None], nk).reshape(-1)
                b32 = g32[k].rule(k, x0[:, None], nk).reshape(-1)
                assert np.abs(b16 - b32).max() < 1e-8
                assert np.abs(val - b32).max() < 2e-6, (k, dd, np.abs(val - b32).max())


def test_far_targets_take_the_near_rule(sphere):
    """At d >= 1.2 h_j the method is the near rule of oracle.nearsing itself."""
    drop, lap, cv, ss, sd = sphere
    x0 = np.array([0.0, 0.6, 0.8]) * (1.0 + 1.5 * ss.h)
    assert np.array_equal(NI.value(ss, x0)[0], ss.upsampled(x0[:, None])[:, 0])
    assert nearsing.UPSAMPLE == 4


def test_near_rule_is_at_rounding_from_two_spacings(sphere):
    """The library applies the four times upsampled rule at every near target; from d = 2 h_j on (the
    workloads keep targets at least 2.6 h_j from other drops) it agrees with the closed forms to rounding."""
    drop, lap, cv, ss, sd = sphere
    rng = np.random.default_rng(6)
    for dd in (2.0, 2.6):
        for _ in range(3):
            v, n0 = _unit(rng), _unit(rng)
            x0 = v * (1.0 + dd * ss.h)
            for n, (c, sl, fl) in lap.items():
                assert abs(float(sl.upsampled(x0[:, None])[0]) - exact_single_layer(n, c, x0)) < 1e-13
                assert abs(float(fl.upsampled(x0[:, None], n0)[0]) - exact_field(n, c, x0) @ n0) < 1e-13
            assert np.abs(ss.upsampled(x0[:, None])[:, 0] - exact_stokeslet_of_constant(cv, x0)).max() < 1e-13
            assert np.abs(sd.upsampled(x0[:, None])[:, 0]).max() < 1e-12
