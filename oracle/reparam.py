"""Reparametrisation of a drop surface (Section 2.2 and the last step of Algorithm 1), plain FP64 numpy
(test infrastructure only).

The paper keeps the spherical-harmonic representation of deforming drops well resolved by a
reparametrisation step and refers to its companion works for the algorithm, which it does not restate.
Reading used here (an optimisation that moves the nodes along the surface while keeping its shape): the
position x(theta, phi) of a drop is moved tangentially to lower the spectral energy

    E(x) = sum over components, degrees n >= 1 and orders m of  n^a |x_nm|^2,

which weights the high-degree content of the parametrisation. One step is an explicit gradient-flow step
whose velocity is the tangential part of the energy gradient, evaluated on the degree-q grid:

    h = sum_{n,m} n^a x_nm Y_nm          (half the gradient of E, as a field on the surface)
    x <- x - tau (h - (h . n) n)         (n the unit normal: only tangential moves)

followed by the Galerkin projection (forward transform, Section 2) of the moved grid positions back to
degree p. A tangential velocity leaves the surface in place to first order in tau; the step is stable for
tau p^a < 1, and tau = c / p^a damps the highest degrees fastest. The unit sphere in the standard
parametrisation is a fixed point (h is then x itself, which is normal).

The surfactant concentration is represented on the same parameter grid, so it moves with the nodes
(Section 2.2 combines the optimisation with the global representation of both the position and the
concentration): the node (theta, phi) now sits where the surface point x - tau t was, t = h - (h . n) n,
and takes the concentration found there, to the same first order,

    Gamma <- Gamma - tau grad_S Gamma . t,   grad_S Gamma . t = [G_a G_b] M^-1 [a . t, b . t]^T,

with the tangents a = x_theta, b = x_phi / sin(theta), their Gram matrix M and G_a, G_b the matching
derivatives of Gamma; the moved values are projected to degree p like the positions.
"""
from __future__ import annotations

import numpy as np

from . import geometry, sh


def degree_weights(p: int, a: float) -> np.ndarray:
    """n^a for every coefficient index n*n + n + m of degree p (0 for n = 0)."""
    w = np.zeros(sh.ncoef(p))
    for n in range(1, p + 1):
        w[n * n:(n + 1) * (n + 1)] = float(n) ** a
    return w


def energy(xcoef, p: int, a: float = 4.0) -> float:
    """E = sum n^a |x_nm|^2 over the three position components."""
    x = np.asarray(xcoef, dtype=np.float64)
    return float((degree_weights(p, a)[None, :] * x * x).sum())


def step(xcoef, p: int, a: float, tau: float, q: int | None = None, gamma=None):
    """One tangential gradient-flow step; returns the new position coefficients (3, (p+1)^2), and with
    `gamma` ((p+1)^2 coefficients) also the transported concentration."""
    q = 2 * p + 1 if q is None else q
    x = np.asarray(xcoef, dtype=np.float64)
    xg, n, _ = geometry.surface_on_grid(x, p, q)
    h = sh.sht_inverse(degree_weights(p, a)[None, :] * x, p, q)
    ht = h - (h * n).sum(axis=0)[None, :] * n
    xnew = sh.sht_forward(xg - tau * ht, p, q)
    if gamma is None:
        return xnew
    S, St, Sp = sh.grid_basis(p, q, derivs=True)
    g = np.asarray(gamma, dtype=np.float64)
    ta, tb = x @ St, x @ Sp                       # tangents a, b (3, N)
    ga, gb = g @ St, g @ Sp
    maa, mab, mbb = (ta * ta).sum(0), (ta * tb).sum(0), (tb * tb).sum(0)
    at, bt = (ta * ht).sum(0), (tb * ht).sum(0)
    det = maa * mbb - mab * mab
    # [G_a G_b] M^-1 [a.t, b.t]^T with M^-1 = [[mbb, -mab], [-mab, maa]] / det
    dg = (ga * (mbb * at - mab * bt) + gb * (maa * bt - mab * at)) / det
    return xnew, sh.sht_forward(g @ S - tau * dg, p, q)


def reparametrize(xcoef, p: int, steps: int = 20, a: float = 4.0, c: float = 0.5, q: int | None = None,
                  gamma=None):
    """`steps` steps of size tau = c / p^a; returns (coefficients, energies before and after each step),
    and with `gamma` (coefficients, energies, transported concentration)."""
    tau = c / float(p) ** a
    x = np.asarray(xcoef, dtype=np.float64)
    g = None if gamma is None else np.asarray(gamma, dtype=np.float64)
    hist = [energy(x, p, a)]
    for _ in range(steps):
        if g is None:
            x = step(x, p, a, tau, q)
        else:
            x, g = step(x, p, a, tau, q, gamma=g)
        hist.append(energy(x, p, a))
    return (x, hist) if g is None else (x, hist, g)
