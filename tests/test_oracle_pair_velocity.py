"""Two drops on the field axis (Section 4.3, multiple drops): the oracle's pair velocity against the h^-2
law of Baygents et al. and against the far field of one drop alone.

Two spherical drops of radius 1 (clean at t = 0: a uniform concentration gives no Marangoni stress) sit
on the z axis with centroids h apart in the uniform field E = z. Each translates along the axis with the
centroid velocity U(h) = (1/V) int x (u.n) dS (Reynolds' transport theorem for the enclosed volume).

* Baygents et al. predict U = O(h^-2): the local slope d ln U / d ln h tends to -2.
* The coefficient follows from the isolated drop. Its exterior flow is axisymmetric and of degree 2,
  with stream function psi = (a + b r^-2) sin^2(theta) cos(theta): a stresslet and a potential
  quadrupole, u_r = 2 (a r^-2 + b r^-4) P_2(cos theta), u_theta = 2 b r^-4 sin(theta) cos(theta). On
  the drop (r = 1) u_r = c_r P_2 and u_theta = c_t sin(theta) cos(theta) fix 2a = c_r - c_t. On the axis
  the flow is (c_r - c_t) h^-2 + O(h^-4), and the other drop moves with it up to relative O(h^-2)
  (Faxen's correction over its size, and the electric interaction of the induced dipoles).

So U(h) h^2 / (c_r - c_t) - 1 = O(h^-2): a check of the drop-to-drop coupling (cross-drop single and
double layers with the (lambda_j - 1) factor, signs, the 1/(4 pi)) against the single-drop solution,
whose normal velocity is Taylor's (tests/test_oracle_physics.py).
"""
import math

import numpy as np
import pytest

import inputs
from oracle import geometry, physics, sh

P_DEG = 6
PRM = physics.Params(R=2.0, Q=0.5, Ca_E=0.1)


def _uniform(p):
    g = np.zeros(sh.ncoef(p))
    g[0] = math.sqrt(4.0 * math.pi)
    return g


def centroid_velocity(xcoef, ucoef, p):
    """(1/V) int x (u.n) dS on the degree 2p+1 grid."""
    q = 2 * p + 1
    sg = physics.SurfaceGrid(xcoef, p, q)
    un = (sg.values(ucoef) * sg.n).sum(axis=0)
    return (sg.x * un * sg.omega * sg.J).sum(axis=1) / geometry.volume(xcoef, p, q)


def surface_modes(ucoef, p):
    """c_r, c_t of a velocity on the unit sphere about the origin and the largest residual of
    u_r - c_r P_2, u_theta - c_t sin cos (the degree-2 axisymmetric form)."""
    q = 2 * p + 1
    th, ph = sh.grid_points(q)
    w = sh.grid_weights(q)
    u = sh.sht_inverse(ucoef, p, q)
    rh = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    thh = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)])
    ur, ut = (u * rh).sum(axis=0), (u * thh).sum(axis=0)
    P2 = 0.5 * (3.0 * np.cos(th) ** 2 - 1.0)
    sc = np.sin(th) * np.cos(th)
    c_r = 5.0 / (4.0 * math.pi) * (w * ur * P2).sum()           # int P_2^2 dOmega = 4 pi / 5
    c_t = (w * ut * sc).sum() / (8.0 * math.pi / 15.0)          # int sin^2 cos^2 dOmega = 8 pi / 15
    return c_r, c_t, max(np.abs(ur - c_r * P2).max(), np.abs(ut - c_t * sc).max())


def pair_velocity(h, lam, p=P_DEG):
    xs = [inputs.sphere_coef(p, centre=(0.0, 0.0, c)) for c in (-0.5 * h, 0.5 * h)]
    u, _ = physics.rates(xs, [_uniform(p)] * 2, [p, p], [lam, lam], PRM, near=True)
    return centroid_velocity(xs[0], u[0], p), centroid_velocity(xs[1], u[1], p)


@pytest.mark.parametrize("lam", [1.0, 3.0])
def test_pair_velocity_follows_the_isolated_drops_far_field(lam):
    p = P_DEG
    u1, _ = physics.rates([inputs.sphere_coef(p)], [_uniform(p)], [p], [lam], PRM, near=True)
    c_r, c_t, resid = surface_modes(u1[0], p)
    assert resid < 1e-12                       # degree 2, axisymmetric
    coef = c_r - c_t
    assert coef > 0.0                          # R > Q: the drops push each other apart along the field
    hs = (12.0, 24.0)
    U = {}
    for h in hs:
        lower, upper = pair_velocity(h, lam)
        # symmetric about the midplane, no motion off the axis (to rounding of the O(0.1) surface
        # velocities the integrals cancel)
        assert abs(lower[2] + upper[2]) < 1e-12
        assert np.abs(upper[:2]).max() < 1e-12
        U[h] = upper[2]
        # the isolated drop's stresslet, up to the relative O(h^-2) corrections
        dev = 1.0 - U[h] * h * h / coef
        assert 1.0 / h ** 2 < dev < 4.0 / h ** 2, (h, dev)
    # Baygents' h^-2 law: the local slope between h = 12 and 24
    slope = math.log(U[24.0] / U[12.0]) / math.log(2.0)
    assert abs(slope + 2.0) < 0.03, slope
    # the correction itself shrinks as h^-2 (a factor of about 4 from 12 to 24)
    r = (1.0 - U[12.0] * 144.0 / coef) / (1.0 - U[24.0] * 576.0 / coef)
    assert 3.0 < r < 5.0, r
