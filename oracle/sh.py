"""Spherical-harmonic machinery of the method, plain FP64 numpy (test infrastructure only).

Follows Section 2 of the paper:
  * Gaussian grid (Eq. spharm_ex): 2q+2 equispaced longitudes phi_k = pi k/(q+1) and q+1
    Gauss-Legendre latitudes theta_j = acos(t_j). Latitudes are ordered by increasing theta
    (t_j decreasing), longitudes by k, values stored [j][k] row-major.
  * Normalised harmonics and Legendre functions with the Condon-Shortley phase
    (Eqs. normalized_spharm, pneg); stored in the real orthonormal basis documented in
    the inputs module (index n*n + n + m).
  * Regular weights: the surface rule of Eq. reg_quadrature written relative to the unit
    sphere, omega_j = (pi/(q+1)) w_j^G (the paper prints pi/p; with 2q+2 longitudes the
    trapezoid spacing is pi/(q+1), which is what makes the weights sum to 4 pi).
  * Forward transform = the Galerkin inner product (y, Y_nm) of Section 2 evaluated with
    that rule; inverse transform = the truncated sum of Eq. spharm_ex.
"""
from __future__ import annotations

import functools
import math

import numpy as np

SQRT2 = math.sqrt(2.0)


def ncoef(p: int) -> int:
    return (p + 1) * (p + 1)


def idx(n: int, m: int) -> int:
    return n * n + n + m


def gauss_grid(q: int):
    """Degree-q Gaussian grid: returns (t, wG, theta, phi) with t decreasing (theta increasing)."""
    x, w = np.polynomial.legendre.leggauss(q + 1)
    t = x[::-1].copy()
    wG = w[::-1].copy()
    theta = np.arccos(t)
    phi = np.pi * np.arange(2 * q + 2) / (q + 1)
    return t, wG, theta, phi


def grid_points(q: int):
    """All nodes of the degree-q grid as flat arrays (theta, phi), [j][k] order."""
    _, _, theta, phi = gauss_grid(q)
    th, ph = np.meshgrid(theta, phi, indexing="ij")
    return th.ravel(), ph.ravel()


def grid_weights(q: int) -> np.ndarray:
    """Regular weights omega per node, [j][k] order: omega_j = (pi/(q+1)) w_j^G."""
    _, wG, _, _ = gauss_grid(q)
    om = (np.pi / (q + 1)) * wG
    return np.repeat(om, 2 * q + 2)


def alf(nmax: int, ct, st):
    """Normalised associated Legendre functions Pbar_n^m(cos theta), 0 <= m <= n <= nmax,
    with the Condon-Shortley phase. ct = cos(theta), st = sin(theta) >= 0 (arrays).
    Returns P with P[n, m] an array shaped like ct (entries with m > n are zero).
    Standard normalised three-term recurrence in n for fixed m, seeded by the sectoral
    values Pbar_m^m = -sqrt((2m+1)/(2m)) sin(theta) Pbar_{m-1}^{m-1}."""
    ct = np.asarray(ct, dtype=np.float64)
    st = np.asarray(st, dtype=np.float64)
    P = np.zeros((nmax + 1, nmax + 1) + ct.shape)
    P[0, 0] = 1.0 / math.sqrt(4.0 * math.pi)
    for m in range(1, nmax + 1):
        P[m, m] = -math.sqrt((2.0 * m + 1.0) / (2.0 * m)) * st * P[m - 1, m - 1]
    for m in range(0, nmax):
        P[m + 1, m] = math.sqrt(2.0 * m + 3.0) * ct * P[m, m]
    for m in range(0, nmax + 1):
        for n in range(m + 2, nmax + 1):
            a = math.sqrt((4.0 * n * n - 1.0) / (n * n - m * m))
            b = math.sqrt(((n - 1.0) ** 2 - m * m) / (4.0 * (n - 1.0) ** 2 - 1.0))
            P[n, m] = a * (ct * P[n - 1, m] - b * P[n - 2, m])
    return P


def _pbar(P, n, m):
    """Pbar_n^m with the negative-order rule Pbar_n^{-1} = -Pbar_n^1 and zero outside range."""
    if m < 0:
        return -P[n, 1] if (m == -1 and n >= 1) else 0.0 * P[0, 0]
    if m > n or n >= P.shape[0]:
        return 0.0 * P[0, 0]
    return P[n, m]


def basis(p: int, ct, st, phi, derivs: bool = False):
    """Real orthonormal harmonics S_nm at points; shape ((p+1)^2, npts).
    With derivs=True also returns dS/dtheta and (1/sin theta) dS/dphi, both computed by
    division-free identities of the normalised Legendre functions:
      d/dtheta Pbar_n^m = (sqrt((n-m)(n+m+1)) Pbar_n^{m+1} - sqrt((n+m)(n-m+1)) Pbar_n^{m-1})/2
      m Pbar_n^m / sin  = -sqrt((2n+1)/(2n+3)) (sqrt((n+m+1)(n+m+2)) Pbar_{n+1}^{m+1}
                                               + sqrt((n-m+1)(n-m+2)) Pbar_{n+1}^{m-1})/2
    so that the result stays accurate at points close to the poles of the chart."""
    ct = np.asarray(ct, dtype=np.float64).ravel()
    st = np.asarray(st, dtype=np.float64).ravel()
    phi = np.asarray(phi, dtype=np.float64).ravel()
    P = alf(p + 1 if derivs else p, ct, st)
    npts = ct.size
    S = np.zeros((ncoef(p), npts))
    if derivs:
        St = np.zeros((ncoef(p), npts))
        Sp = np.zeros((ncoef(p), npts))
    for n in range(p + 1):
        for m in range(0, n + 1):
            pv = P[n, m]
            if derivs:
                if m == 0:
                    dth = math.sqrt(n * (n + 1.0)) * _pbar(P, n, 1)
                    msin = 0.0 * pv
                else:
                    dth = 0.5 * (math.sqrt((n - m) * (n + m + 1.0)) * _pbar(P, n, m + 1)
                                 - math.sqrt((n + m) * (n - m + 1.0)) * _pbar(P, n, m - 1))
                    msin = -0.5 * math.sqrt((2.0 * n + 1.0) / (2.0 * n + 3.0)) * (
                        math.sqrt((n + m + 1.0) * (n + m + 2.0)) * _pbar(P, n + 1, m + 1)
                        + math.sqrt((n - m + 1.0) * (n - m + 2.0)) * _pbar(P, n + 1, m - 1))
            if m == 0:
                S[idx(n, 0)] = pv
                if derivs:
                    St[idx(n, 0)] = dth
                    Sp[idx(n, 0)] = 0.0
            else:
                c = np.cos(m * phi)
                s = np.sin(m * phi)
                S[idx(n, m)] = SQRT2 * pv * c
                S[idx(n, -m)] = SQRT2 * pv * s
                if derivs:
                    St[idx(n, m)] = SQRT2 * dth * c
                    St[idx(n, -m)] = SQRT2 * dth * s
                    Sp[idx(n, m)] = -SQRT2 * msin * s
                    Sp[idx(n, -m)] = SQRT2 * msin * c
    if derivs:
        return S, St, Sp
    return S


@functools.lru_cache(maxsize=16)
def grid_basis(p: int, q: int, derivs: bool = False):
    """Basis (and derivatives) of degree p on all nodes of the degree-q grid (cached; the
    returned arrays are shared and must not be modified)."""
    th, ph = grid_points(q)
    out = basis(p, np.cos(th), np.sin(th), ph, derivs=derivs)
    for a in (out if derivs else (out,)):
        a.setflags(write=False)
    return out


def sht_inverse(coef, p: int, q: int) -> np.ndarray:
    """Eq. spharm_ex: values of the degree-p expansion on the degree-q grid.
    coef (..., (p+1)^2) -> (..., (q+1)(2q+2))."""
    S = grid_basis(p, q)
    return np.asarray(coef) @ S


def sht_forward(vals, p: int, q: int) -> np.ndarray:
    """Galerkin inner products (y, S_nm) by the regular rule on the degree-q grid.
    vals (..., (q+1)(2q+2)) -> (..., (p+1)^2)."""
    S = grid_basis(p, q)
    om = grid_weights(q)
    return (np.asarray(vals) * om) @ S.T


def legendre_sum(q: int, t) -> np.ndarray:
    """sum_{n=0}^{q} P_n(t) for unnormalised Legendre polynomials (Bonnet recurrence)."""
    t = np.asarray(t, dtype=np.float64)
    p0 = np.ones_like(t)
    p1 = t.copy()
    tot = p0 + (p1 if q >= 1 else 0.0)
    for n in range(1, q):
        p2 = ((2.0 * n + 1.0) * t * p1 - n * p0) / (n + 1.0)
        tot = tot + p2
        p0, p1 = p1, p2
    return tot
