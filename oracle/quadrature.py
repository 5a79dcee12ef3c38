"""Regular and singular quadrature of the layer kernels, plain FP64 numpy (test infrastructure only).

Kernels (Eqs. GandT, op_stokes, dl_op_laplace), xh = x0 - x, r = |xh|, all with the 1/(4 pi)
of the operator definitions:
    'lsl'   Laplace single layer        sigma / r
    'ladl'  Laplace double layer of Eq. E_n, normal at the target x0:
                                          sigma (xh . n(x0)) / r^3
    'sto_s' Stokeslet                    f . G,  G = I/r + xh xh / r^3
    'sto_d' stresslet with source normal u . T . n(x),  T = -6 xh xh xh / r^5

Regular rule (Eq. reg_quadrature) on the degree-q source grid: int y dS = sum omega_j y J.

Singular self-integration (Section 2.1, Eq. mod_weights): the parametrisation is rotated so
that the target is the north pole, and the rotated grid is summed with the modified weights
    mu_j = omega_j * 2 sin(theta_j / 2) * sum_{n=0}^{q} P_n(cos theta_j),
which integrate g / |north pole - y| exactly for g of degree <= q on the unit sphere
(generating function of the Legendre polynomials). The oracle rotates by evaluating the
original expansions directly at the rotated points (no rotation of coefficients).
The rotation used for target direction (theta0, phi0) is R = Rz(phi0) Ry(theta0).
"""
from __future__ import annotations

import math

import numpy as np

from . import geometry, sh

INV4PI = 1.0 / (4.0 * math.pi)


def modified_weights(q: int) -> np.ndarray:
    """mu per node of the degree-q grid ([j][k] order)."""
    t, wG, theta, _ = sh.gauss_grid(q)
    mu = (np.pi / (q + 1)) * wG * 2.0 * np.sin(0.5 * theta) * sh.legendre_sum(q, t)
    return np.repeat(mu, 2 * q + 2)


def _rz(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rotation(theta0: float, phi0: float, gamma: float = 0.0) -> np.ndarray:
    """Rz(phi0) Ry(theta0) Rz(gamma): takes the north pole to direction (theta0, phi0).
    gamma (spin about the pole) is free; the method's result depends on it only through
    the quadrature error."""
    cy, sy = math.cos(theta0), math.sin(theta0)
    Ry = np.array([[cy, 0.0, sy], [0.0, 1.0, 0.0], [-sy, 0.0, cy]])
    return _rz(phi0) @ Ry @ _rz(gamma)


def unit_grid(q: int) -> np.ndarray:
    th, ph = sh.grid_points(q)
    return np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])


# ---------------------------------------------------------------- pointwise kernels

def kernel_scalar(kind: str, x0, n0, x):
    """Scalar Laplace kernels for one target x0 (3,) against points x (3,N)."""
    xh = x0[:, None] - x
    r2 = (xh * xh).sum(axis=0)
    r = np.sqrt(r2)
    if kind == "lsl":
        return 1.0 / r
    if kind == "ladl":
        return (xh * n0[:, None]).sum(axis=0) / (r2 * r)
    raise ValueError(kind)


def kernel_tensor(kind: str, x0, x, n):
    """Stokes kernels as 3x3 matrices acting on the density: out_i = K_ik rho_k; (3,3,N)."""
    xh = x0[:, None] - x
    r2 = (xh * xh).sum(axis=0)
    r = np.sqrt(r2)
    if kind == "sto_s":
        K = xh[:, None, :] * xh[None, :, :] / (r2 * r)
        K = K + np.eye(3)[:, :, None] / r
        return K
    if kind == "sto_d":
        xn = (xh * n).sum(axis=0)
        return -6.0 * xh[:, None, :] * xh[None, :, :] * xn / (r2 * r2 * r)
    raise ValueError(kind)


# ---------------------------------------------------------------- regular sums

def regular_scalar(kind: str, x0, n0, xs, ws, dens):
    """(1/4pi) sum_s K(x0_t, xs_s) ws_s dens_s for every target t. x0,n0 (3,T)."""
    out = np.zeros(x0.shape[1])
    for t in range(x0.shape[1]):
        out[t] = (kernel_scalar(kind, x0[:, t], n0[:, t], xs) * ws * dens).sum()
    return INV4PI * out


def regular_tensor(kind: str, x0, xs, ns, ws, dens):
    """(1/4pi) sum_s K(x0_t, xs_s) . dens_s ws_s; dens (3,S) -> (3,T)."""
    out = np.zeros((3, x0.shape[1]))
    for t in range(x0.shape[1]):
        K = kernel_tensor(kind, x0[:, t], xs, ns)
        out[:, t] = np.einsum("iks,ks->i", K, dens * ws)
    return INV4PI * out


# ---------------------------------------------------------------- singular self rows

def self_rows(xcoef, p: int, q: int, theta0: float, phi0: float, kinds, gamma: float = 0.0):
    """Rows of the singular self-integration for one target at parameter (theta0, phi0).

    Returns {kind: row}: scalar kinds give row (ncoef,) with value = row . sigma_coef;
    tensor kinds give row (3,3,ncoef) with value_i = sum_k row[i,k] . dens_coef[k]."""
    R = rotation(theta0, phi0, gamma)
    P = R @ unit_grid(q)
    ct = P[2]
    st = np.hypot(P[0], P[1])
    ph = np.arctan2(P[1], P[0])
    x, n, J = geometry.surface_at(xcoef, p, ct, st, ph)
    S = sh.basis(p, ct, st, ph)
    x0, n0, _ = geometry.surface_at(xcoef, p, np.array([math.cos(theta0)]),
                                    np.array([math.sin(theta0)]), np.array([phi0]))
    x0 = x0[:, 0]
    n0 = n0[:, 0]
    w = modified_weights(q) * J * INV4PI
    out = {}
    for kind in kinds:
        if kind in ("lsl", "ladl"):
            out[kind] = S @ (w * kernel_scalar(kind, x0, n0, x))
        else:
            K = kernel_tensor(kind, x0, x, n)
            out[kind] = np.einsum("iks,cs->ikc", K * w, S)
    return out
