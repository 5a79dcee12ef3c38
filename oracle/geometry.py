"""Surface geometry from position coefficients, plain FP64 numpy (test infrastructure only).

Each position component is a degree-p expansion (Section 2, Eq. spharm_ex). At any
parameter point the oracle evaluates x, the tangents x_theta and x_phi/sin(theta), and
    c = x_theta x (x_phi / sin theta),   J = |c|,   n = c / J,
so J is the area element relative to the unit sphere (W / sin theta with W the element of
Eq. reg_quadrature) and n the outward unit normal of Section 1 (for the standard
orientation, where the unit sphere gives J = 1 and n = x).
"""
from __future__ import annotations

import numpy as np

from . import sh


def surface_at(xcoef, p: int, ct, st, phi):
    """x (3,N), n (3,N), J (N,) at parameter points given by cos/sin theta and phi."""
    S, St, Sp = sh.basis(p, ct, st, phi, derivs=True)
    xcoef = np.asarray(xcoef, dtype=np.float64)
    x = xcoef @ S
    xt = xcoef @ St
    xps = xcoef @ Sp
    c = np.cross(xt.T, xps.T).T
    J = np.sqrt((c * c).sum(axis=0))
    n = c / J
    return x, n, J


def surface_on_grid(xcoef, p: int, q: int):
    """Geometry on every node of the degree-q grid ([j][k] order)."""
    th, ph = sh.grid_points(q)
    return surface_at(xcoef, p, np.cos(th), np.sin(th), ph)


def area(xcoef, p: int, q: int) -> float:
    _, _, J = surface_on_grid(xcoef, p, q)
    return float((sh.grid_weights(q) * J).sum())


def volume(xcoef, p: int, q: int) -> float:
    """Enclosed volume by the divergence theorem, (1/3) int x . n dS."""
    x, n, J = surface_on_grid(xcoef, p, q)
    return float((sh.grid_weights(q) * J * (x * n).sum(axis=0)).sum() / 3.0)
