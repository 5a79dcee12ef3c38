"""Pins of the oracle's reparametrisation (Section 2.2, Algorithm 1): the nodes move along the surface,
so the surface stays where it is, and the spectral energy of the parametrisation goes down."""
import math

import numpy as np
import pytest

import inputs
from oracle import geometry, reparam, sh


def _distorted_sphere(p, eps=0.08):
    """The unit sphere with its parameter points moved along the sphere by a wavy tangential field,
    x = normalise(s + eps grad_S(Y)) with Y = sin^6(theta) cos(6 phi) (degree-6 content), projected to
    degree p: the same surface, a parametrisation with high-degree content."""
    q = 2 * p + 1
    th, ph = sh.grid_points(q)
    s = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    e_th = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)])
    e_ph = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)])
    dth = 6 * np.sin(th) ** 5 * np.cos(th) * np.cos(6 * ph)
    dph = -6 * np.sin(th) ** 5 * np.sin(6 * ph)     # (1/sin) d/dphi of sin^6 cos(6 phi)
    x = s + eps * (dth * e_th + dph * e_ph)
    x = x / np.linalg.norm(x, axis=0)
    return sh.sht_forward(x, p, q)


def _high_energy(x, p, n0):
    w = np.array([1.0 if n >= n0 else 0.0 for n in range(p + 1) for _ in range(2 * n + 1)])
    return float((w[None, :] * x * x).sum())


def test_unit_sphere_is_a_fixed_point():
    p = 8
    x0 = inputs.sphere_coef(p)
    x1, hist = reparam.reparametrize(x0, p, steps=5)
    assert np.abs(x1 - x0).max() < 1e-12
    assert abs(hist[-1] - hist[0]) < 1e-12 * hist[0]


def _off_sphere(x, p):
    xf, _, _ = geometry.surface_on_grid(x, p, 3 * p)
    return float(np.abs(np.linalg.norm(xf, axis=0) - 1).max())


def test_distorted_sphere_keeps_its_surface_and_loses_energy():
    """The flow is tangential, so the explicit steps leave the surface only at second order in the step:
    for the same pseudo-time, halving tau halves how far the nodes leave the sphere and the volume drift
    (a dropped normal projection would move the surface at first order and fail the fixed-point pin)."""
    p = 16
    x0 = _distorted_sphere(p, eps=0.01)
    v0, d0 = geometry.volume(x0, p, 2 * p + 1), _off_sphere(x0, p)
    assert d0 < 2e-6 and abs(v0 - 4 * math.pi / 3) < 1e-7         # a sphere, badly parametrised
    drift = []
    for c, steps in ((1.0, 40), (0.5, 80)):
        x1, hist = reparam.reparametrize(x0, p, steps=steps, c=c)
        assert all(b < a for a, b in zip(hist, hist[1:]))         # energy decreases every step
        assert _high_energy(x1, p, 5) < 0.25 * _high_energy(x0, p, 5)   # the high-degree content goes
        drift.append((abs(geometry.volume(x1, p, 2 * p + 1) - v0), _off_sphere(x1, p)))
    assert drift[0][0] < 1e-4 and drift[0][1] < 5e-5
    assert drift[1][0] < 0.6 * drift[0][0] and drift[1][1] < 0.7 * drift[0][1], drift


def test_perturbed_drop_keeps_volume_and_area():
    p = 10
    x0 = inputs.perturbed_coef(p, np.random.default_rng(3), 1.0, (0.2, -0.1, 0.3))
    v0, a0 = geometry.volume(x0, p, 2 * p + 1), geometry.area(x0, p, 2 * p + 1)
    x1, hist = reparam.reparametrize(x0, p, steps=20)
    assert hist[-1] < hist[0]
    dv = abs(geometry.volume(x1, p, 2 * p + 1) - v0)
    assert dv < 1e-6 * v0
    assert abs(geometry.area(x1, p, 2 * p + 1) - a0) < 1e-6 * a0
    x2, _ = reparam.reparametrize(x0, p, steps=40, c=0.25)       # same pseudo-time, half the step
    assert abs(geometry.volume(x2, p, 2 * p + 1) - v0) < 0.6 * dv


def test_concentration_follows_the_nodes():
    """A concentration that is a function of position, Gamma = z on the surface, must stay that function:
    grad_S z . t is the z component of the tangential move, so the transported Gamma equals the new z
    coordinate exactly (a wrong metric inverse, a swapped tangent or a sign error breaks the identity).
    The total amount int Gamma dS stays put to the degree-p truncation of the moved values (a
    concentration left behind on the old nodes changes it by a thousand times more here)."""
    p = 10
    x0 = inputs.perturbed_coef(p, np.random.default_rng(5), 1.0, (0.1, 0.2, -0.3))
    x1, _, g1 = reparam.reparametrize(x0, p, steps=15, gamma=x0[2].copy())
    assert np.abs(g1 - x1[2]).max() < 1e-12 * np.abs(x1[2]).max()
    q = 2 * p + 1
    om = sh.grid_weights(q)
    g0 = 1.0 + 0.3 * x0[0] / np.abs(x0[0]).max()                 # a positive concentration
    mass = lambda x, g: float((om * geometry.surface_on_grid(x, p, q)[2] * sh.sht_inverse(g, p, q)).sum())
    m0 = mass(x0, g0)
    xa, _, ga = reparam.reparametrize(x0, p, steps=15, c=0.5, gamma=g0)
    assert abs(mass(xa, ga) - m0) < 1e-5 * abs(m0)
    assert abs(mass(xa, g0) - m0) > 1e-3 * abs(m0)               # not transporting would show
