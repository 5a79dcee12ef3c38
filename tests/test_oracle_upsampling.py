"""Pins of the adaptive upsampling reading (oracle/upsampling.py, Section 2): the mean curvature against a
closed form, the aliasing estimate against the measured aliasing of the degree-p projection of H, and the
chosen degree against the tolerance it is asked for.

Closed form: the spheroid x = (a sin t cos f, a sin t sin f, c cos t) (degree 1 in the harmonics) has,
with s^2 = a^2 cos^2 t + c^2 sin^2 t, the principal curvatures a c / s^3 (meridian) and c / (a s)
(parallel), so H = (c / (2 a s)) (1 + a^2 / s^2), 1 on the unit sphere (the oracle's sign).
"""
import numpy as np
import pytest

import inputs
from oracle import physics, sh, upsampling as U


def spheroid(p, a, c):
    x = inputs.sphere_coef(p)
    x[0] *= a
    x[1] *= a
    x[2] *= c
    return x


def h_spheroid(a, c, theta):
    s = np.sqrt(a * a * np.cos(theta) ** 2 + c * c * np.sin(theta) ** 2)
    return c / (2.0 * a * s) * (1.0 + a * a / (s * s))


def true_aliasing(x, p, q, q_ref):
    """Relative error of the degree-p projection of H formed on the degree-q grid, against the
    projection on a degree-q_ref grid."""
    ref = sh.sht_forward(physics.SurfaceGrid(x, p, q_ref).H, p, q_ref)
    got = sh.sht_forward(physics.SurfaceGrid(x, p, q).H, p, q)
    return np.linalg.norm(got - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("c", [0.6, 1.0, 2.0])
def test_mean_curvature_of_spheroids(c):
    p = 6
    sg = physics.SurfaceGrid(spheroid(p, 1.0, c), p, 2 * p + 1)
    np.testing.assert_allclose(sg.H, h_spheroid(1.0, c, sg.theta), rtol=0, atol=1e-13)


def test_sphere_needs_no_upsampling():
    p = 8
    assert U.adaptive_degree(inputs.sphere_coef(p), p, 1e-14) == p


@pytest.mark.parametrize("c", [1.5, 2.0, 3.0])
def test_estimate_tracks_the_measured_aliasing_of_spheroids(c):
    """The estimate is within a factor 4 of the measured aliasing wherever that is above rounding."""
    p = 8
    x = spheroid(p, 1.0, c)
    E = U.curvature_spectrum(x, p, 2 * p + 1)
    for q in (p, 12, 2 * p + 1, 24):
        t = true_aliasing(x, p, q, 10 * p)
        if t > 1e-12:
            e = U.aliasing_estimate(E, p, q)
            assert t / 4.0 < e < 4.0 * t, (q, e, t)


def test_chosen_degree_meets_the_tolerance():
    """On spheroids and a perturbed drop of the workloads' recipe, the degree chosen for eps leaves a
    measured aliasing below 4 eps; more elongated spheroids need more upsampling."""
    p = 8
    rng = np.random.default_rng(0)
    shapes = [spheroid(p, 1.0, c) for c in (1.2, 1.5, 2.0)] + [inputs.perturbed_coef(p, rng, 1.0, (0.0, 0.0, 0.0))]
    for eps in (1e-6, 1e-10):
        qs = []
        for x in shapes:
            q = U.adaptive_degree(x, p, eps)
            assert true_aliasing(x, p, q, 10 * p) < 4.0 * eps, (q, eps)
            qs.append(q)
        assert qs[0] < qs[1] < qs[2]


def test_workload_shapes_at_the_fixed_grid():
    """The library forms the nonlinear terms on the fixed degree 2p+1 grid. For drops of the workloads'
    recipe the adaptive rule at eps = 1e-10 asks for about that at p = 16 and for less at p = 32; the
    measured aliasing of the fixed grid at p = 16 is about 1e-10."""
    rng = np.random.default_rng(0)
    x16 = inputs.perturbed_coef(16, rng, 1.0, (0.0, 0.0, 0.0))
    assert abs(U.adaptive_degree(x16, 16, 1e-10) - 33) <= 2
    assert true_aliasing(x16, 16, 33, 96) < 3e-10
    x32 = inputs.perturbed_coef(32, rng, 1.0, (0.0, 0.0, 0.0))
    assert U.adaptive_degree(x32, 32, 1e-10) < 2 * 32 + 1
