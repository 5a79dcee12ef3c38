"""Pins of the fast all-target rotation (oracle/fastrot.py, Section 2.1): the non-uniform FFT against the
trigonometric sum it evaluates, the rotated values of all targets of a latitude against evaluation at the
rotated points, and the singular rule built on them against oracle.quadrature's rows."""
import math

import numpy as np
import pytest

import inputs
from oracle import fastrot as F, operators, quadrature, sh


def test_nufft_matches_the_trigonometric_sum():
    rng = np.random.default_rng(0)
    M = 34
    B = rng.standard_normal((3, M)) + 1j * rng.standard_normal((3, M))
    x = rng.uniform(-1.0, 8.0, 50)
    s = np.fft.fftfreq(M, 1.0 / M)
    direct = B @ np.exp(1j * s[:, None] * x[None, :])
    got = F.nufft2(B, x)
    assert np.abs(got - direct).max() < 1e-13 * np.abs(B).sum(axis=1).max()


@pytest.mark.parametrize("p", [4, 9])
def test_rotated_values_of_a_latitude_match_direct_evaluation(p):
    """Every target l of two latitudes of the degree-p grid, R = Rz(2 pi l / L) Ry(theta0), L = 2p + 2,
    on the degree 2p + 1 rotated grid; also a coefficient set of degree above L/2 (folded longitudes)."""
    rng = np.random.default_rng(p)
    q, L = 2 * p + 1, 2 * p + 2
    _, _, thetas, _ = sh.gauss_grid(p)
    for deg in (p, 2 * p + 1):
        coef = rng.standard_normal(sh.ncoef(deg))
        for th0 in (thetas[0], thetas[p // 2]):
            fast = F.rotated_values(coef, deg, q, th0, L)
            for l in range(L):
                P = quadrature.rotation(th0, 2.0 * math.pi * l / L) @ quadrature.unit_grid(q)
                direct = coef @ sh.basis(deg, P[2], np.hypot(P[0], P[1]), np.arctan2(P[1], P[0]))
                assert np.abs(fast[l] - direct).max() < 1e-13 * np.abs(coef).sum()


@pytest.mark.parametrize("kind", ["lsl", "ladl", "sto_s", "sto_d"])
def test_singular_rule_through_the_fast_rotation(kind):
    """The rotated-pole rule (Eq. mod_weights) at every target of a perturbed drop from the fast rotated
    values equals the oracle's rows (direct evaluation at each target's rotated points) to 1e-12."""
    p = 5
    rng = np.random.default_rng(11)
    xc = inputs.perturbed_coef(p, rng, 1.0, (0.3, -0.2, 0.1))
    drop = operators.DropGeom(xc, p, 1.0)
    if kind in ("lsl", "ladl"):
        dens = inputs.random_density(p, rng, 1).ravel()
        ref = drop.rows(kind) @ dens
    else:
        dens = inputs.random_density(p, rng, 3)
        ref = np.einsum("tikc,kc->it", drop.rows(kind), dens)
    got = F.self_values(xc, p, dens, kind)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
