"""Adaptive upsampling from the decay of the mean curvature's spectrum, plain FP64 numpy (test
infrastructure only).

Section 2: the geometric quantities built by nonlinear operations (normals, the mean curvature H, the
interfacial force) are formed on a finer grid than the degree-p representation and projected back to
degree p (de-aliasing); the upsampling rate is chosen adaptively from how fast the spectrum of H decays
(the paper refers to Rahimian et al. for the algorithm and states no parameters). The reading used here
ties the rate to the error it controls, the aliasing of the Galerkin projection onto degree p:

  * the regular rule of the degree-q Gauss grid integrates H Y_nm (n <= p) exactly when H has degree
    <= 2q + 1 - p, so the projection of H computed on that grid errs by about the part of H above
    degree 2q + 1 - p;
  * the spectrum E_n = sum_m H_nm^2 is computed once on the probe grid of degree q_s = 2p + 1 (H from
    the exact derivatives of the position expansion); above degree q_s it is extrapolated with the
    geometric decay E_n ~ C rho^n fitted (least squares on log E_n) over the degrees p + 1 .. q_s;
  * the estimated aliasing error of q is sqrt(sum_{n >= 2q + 2 - p} E_n) / |H|_2 (measured E_n up to
    q_s, extrapolated above), and the upsampled degree is the smallest q >= p below the tolerance eps.
A sphere gives q = p (H is constant).
"""
from __future__ import annotations

import math

import numpy as np

from . import sh
from .physics import SurfaceGrid


def curvature_spectrum(xcoef, p: int, q: int) -> np.ndarray:
    """E_n, n = 0..q, of H computed on the degree-q grid."""
    c = sh.sht_forward(SurfaceGrid(xcoef, p, q).H, q, q)
    return np.array([float((c[n * n:(n + 1) * (n + 1)] ** 2).sum()) for n in range(q + 1)])


def aliasing_estimate(E: np.ndarray, p: int, q: int) -> float:
    """Estimated relative error of the degree-p projection of H formed on the degree-q grid, from the
    probe spectrum E (degrees 0..q_s) and its geometric extrapolation."""
    qs = E.size - 1
    total = float(E.sum())
    n0 = 2 * q + 2 - p
    tail = float(E[min(n0, qs + 1):].sum())
    ns = np.arange(p + 1, qs + 1)
    En = E[p + 1:]
    ok = En > 1e-28 * total                       # rounding noise (a sphere) carries no decay
    if ok.sum() >= 2:
        b, a = np.polyfit(ns[ok], np.log(En[ok]), 1)
        rho = math.exp(min(b, -1e-3))               # a spectrum that does not decay counts as barely decaying
        first = max(n0, qs + 1)
        tail += math.exp(a) * rho ** first / (1.0 - rho)
    return math.sqrt(tail / total)


def adaptive_degree(xcoef, p: int, eps: float = 1e-12, q_max: int | None = None) -> int:
    """The smallest q >= p whose estimated aliasing error is below eps (q_max, default 8p + 7, if none)."""
    q_max = 8 * p + 7 if q_max is None else q_max
    E = curvature_spectrum(xcoef, p, 2 * p + 1)
    for q in range(p, q_max + 1):
        if aliasing_estimate(E, p, q) < eps:
            return q
    return q_max
