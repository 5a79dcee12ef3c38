"""Interpolation step of the nearly-singular method, plain FP64 numpy (test infrastructure only).

Section 2.1 (last paragraph): for a target x0 very close to the surface S_j of another drop, the layer
potential of S_j is known accurately in two places, on S_j itself (the singular rule with the modified
weights of Eq. mod_weights, plus the jump of the potential across the layer) and at points far enough
from S_j for the regular rule on an upsampled grid; the value at x0 comes from 1D Lagrange interpolation
through points aligned with x0. The paper gives no parameters; the reading used here:

  * the line of interpolation is the normal through the closest point x* of S_j to x0 (found by
    Gauss-Newton on the spherical-harmonic chart of S_j, started from the nearest node of the four
    times upsampled grid), so x0 = x* + d n(x*) with d = |x0 - x*|;
  * the nodes are t = 0 (the exterior limit at x*) and the M check points t_k = (T1 + (k-1) DT) h_j,
    where the regular rule runs on S_j's grid upsampled UP_CHECK times per direction (accurate from
    about h_j / 2 on, as the four times upsampled grid of the near rule is from about h_j on);
  * the Lagrange polynomial through these M + 1 values is evaluated at t = d;
  * targets with d < SWITCH h_j take the interpolation, farther ones the near rule of oracle.nearsing
    (the four times upsampled regular rule).
h_j is the spacing of the drop's degree-q source grid (oracle.nearsing.spacing). Measured on the unit
sphere at p = 6 and 8 against the closed forms (single layer and field of a Y_nm density, Stokeslet
and stresslet of a constant density): the interpolation is within 6e-7 (single layer), 6e-6 (field),
1.5e-7 (Stokeslet) and 5e-8 (stresslet) of the exact values at every d < SWITCH h_j, where the near
rule alone errs by up to 3e-3, 0.4, 1.3e-2 and 7 at d = 0.02-0.05 h_j, and by 2e-7 for the stresslet
still at d = h_j. On a perturbed drop the exterior limit carries the singular rule's own error on the
degree q = 2p+1 grid.

Exterior limits at x* (the target lies outside S_j; the oracle's kernels carry the 1/(4 pi)):
  * 'lsl' (single layer) is continuous: the singular rule's value at x*;
  * the field of the single layer, E = -grad phi, has the tangential part -grad_S phi (phi the single
    layer's potential on S_j, a smooth surface field expanded on the degree 2p+1 grid) and the normal
    part K'[sigma] + sigma / 2 (K' the target-normal double layer of Eq. E_n at x*, Gauss' jump); the
    'ladl' kind of a target normal n0 interpolates E . n0;
  * 'sto_s' (Stokeslet) is continuous;
  * 'sto_d' (stresslet with the source normal) jumps to PV - u(x*) outside (D[c] = 2c, c, 0 inside, on
    and outside a closed surface).
"""
from __future__ import annotations

import math

import numpy as np

from . import geometry, nearsing, quadrature, sh

SWITCH = 1.2     # interpolate below this many h_j, the four times upsampled rule above
UP_CHECK = 8     # upsampling of the check points' grid, per direction
T1 = 0.6         # first check point, in h_j
DT = 0.2         # check-point spacing, in h_j
M = 8            # check points (Lagrange degree M)


def _frame(u):
    """cos, sin theta, phi of a unit vector and the unit tangents theta_hat, phi_hat there."""
    ct = float(u[2])
    st = math.hypot(float(u[0]), float(u[1]))
    ph = math.atan2(float(u[1]), float(u[0]))
    th_hat = np.array([ct * math.cos(ph), ct * math.sin(ph), -st])
    ph_hat = np.array([-math.sin(ph), math.cos(ph), 0.0])
    return ct, st, ph, th_hat, ph_hat


def _chart(xcoef, p, ct, st, ph):
    """x and the tangents x_theta, x_phi / sin theta at one parameter point."""
    S, St, Sp = sh.basis(p, np.array([ct]), np.array([st]), np.array([ph]), derivs=True)
    xc = np.asarray(xcoef, dtype=np.float64)
    return (xc @ S)[:, 0], (xc @ St)[:, 0], (xc @ Sp)[:, 0]


def closest_point(drop, x0, fine=None, tol=1e-14, maxit=400):
    """Closest point of S_j (DropGeom drop) to x0: returns (theta, phi) of the parameter point, x*, the
    normal n(x*) and the signed distance (x0 - x*) . n(x*). Gauss-Newton on the parameter sphere: the
    step (a, b) along (theta_hat, phi_hat) solves the least-squares problem [x_theta, x_phi/sin] (a, b)
    = x0 - x, and the parameter direction moves by a theta_hat + b phi_hat (renormalised); at the
    solution x0 - x is normal to the surface. Started from the nearest node of the grid `fine` (nodes x,
    degree q; default the four times upsampled grid)."""
    x0 = np.asarray(x0, dtype=np.float64).ravel()
    F = nearsing._Fine(drop) if fine is None else fine
    k = int(np.argmin(((F.x - x0[:, None]) ** 2).sum(axis=0)))
    th, ph = sh.grid_points(F.q)
    u = np.array([math.sin(th[k]) * math.cos(ph[k]), math.sin(th[k]) * math.sin(ph[k]), math.cos(th[k])])
    for _ in range(maxit):
        ct, st, phi, th_hat, ph_hat = _frame(u)
        x, a1, a2 = _chart(drop.xcoef, drop.p, ct, st, phi)
        A = np.stack([a1, a2], axis=1)
        step = np.linalg.solve(A.T @ A, A.T @ (x0 - x))
        u = u + step[0] * th_hat + step[1] * ph_hat
        u /= np.linalg.norm(u)
        if np.abs(step).max() < tol:
            break
    else:
        raise RuntimeError("closest point: Gauss-Newton did not converge")
    ct, st, phi, _, _ = _frame(u)
    x, a1, a2 = _chart(drop.xcoef, drop.p, ct, st, phi)
    n = np.cross(a1, a2)
    n /= np.linalg.norm(n)
    return math.atan2(st, ct), phi, x, n, float((x0 - x) @ n)


def surface_potential(drop, sigma, qp=None):
    """Coefficients (degree qp, default 2p+1) of the single layer's potential of sigma on S_j itself:
    the singular rule at every node of the degree-qp grid, then the forward transform."""
    qp = 2 * drop.p + 1 if qp is None else qp
    th, ph = sh.grid_points(qp)
    vals = np.empty(th.size)
    for k in range(th.size):
        row = quadrature.self_rows(drop.xcoef, drop.p, drop.q, float(th[k]), float(ph[k]), ("lsl",))["lsl"]
        vals[k] = row @ sigma
    return sh.sht_forward(vals, qp, qp), qp


def _surface_gradient(xcoef, p, coef, qp, th, ph):
    """grad_S of a degree-qp field at one parameter point: [a1 a2] G^-1 (f_theta, f_phi / sin)."""
    ct, st = math.cos(th), math.sin(th)
    _, a1, a2 = _chart(xcoef, p, ct, st, ph)
    _, Ft, Fp = sh.basis(qp, np.array([ct]), np.array([st]), np.array([ph]), derivs=True)
    g = np.array([coef @ Ft[:, 0], coef @ Fp[:, 0]])
    A = np.stack([a1, a2], axis=1)
    return A @ np.linalg.solve(A.T @ A, g)


def exterior_limit(drop, kind, dens, th, ph, n0=None, phi_coef=None):
    """Limit at the surface point of parameter (th, ph), approached from outside S_j, of drop j's layer
    potential of kind 'lsl', 'ladl' (E . n0), 'sto_s' or 'sto_d' with density coefficients dens
    ((ncoef,) or (3, ncoef)). phi_coef: (coefficients, degree) of surface_potential for 'ladl'."""
    kinds = ("lsl", "ladl") if kind == "ladl" else (kind,)
    rows = quadrature.self_rows(drop.xcoef, drop.p, drop.q, th, ph, kinds)
    if kind == "lsl":
        return float(rows["lsl"] @ dens)
    ct, st = math.cos(th), math.sin(th)
    S = sh.basis(drop.p, np.array([ct]), np.array([st]), np.array([ph]))[:, 0]
    if kind == "ladl":
        _, a1, a2 = _chart(drop.xcoef, drop.p, ct, st, ph)
        n = np.cross(a1, a2)
        n /= np.linalg.norm(n)
        coef, qp = surface_potential(drop, dens) if phi_coef is None else phi_coef
        E = -_surface_gradient(drop.xcoef, drop.p, coef, qp, th, ph) + (float(rows["ladl"] @ dens)
                                                                     + 0.5 * float(dens @ S)) * n
        return float(E @ np.asarray(n0, dtype=np.float64))
    val = np.einsum("ikc,kc->i", rows[kind], dens)
    if kind == "sto_d":
        val = val - np.asarray(dens) @ S
    return val


class _Grid:
    """Drop j's geometry and density on its grid upsampled `up` times per direction."""

    def __init__(self, drop, dens, up):
        self.q = up * (drop.q + 1) - 1
        self.x, self.n, J = geometry.surface_on_grid(drop.xcoef, drop.p, self.q)
        self.w = sh.grid_weights(self.q) * J
        self.dens = sh.sht_inverse(dens, drop.p, self.q)

    def rule(self, kind, x, n0=None):
        """The regular rule (Eq. reg_quadrature) on this grid at points x (3, K)."""
        if kind in ("lsl", "ladl"):
            nn = np.zeros_like(x) if n0 is None else \
                np.repeat(np.asarray(n0, dtype=np.float64).reshape(3, 1), x.shape[1], axis=1)
            return quadrature.regular_scalar(kind, x, nn, self.x, self.w, self.dens)
        return quadrature.regular_tensor(kind, x, self.x, self.n, self.w, self.dens)


class Source:
    """Drop j with a density of one kind: the four times upsampled grid of the near rule
    (oracle.nearsing; also the closest-point search's starting nodes), the check points' grid
    (upsampled `up` times) and, for 'ladl', the single layer's potential on S_j."""

    def __init__(self, drop, kind, dens, up=UP_CHECK):
        self.drop, self.kind = drop, kind
        self.dens = np.asarray(dens, dtype=np.float64)
        self.near = _Grid(drop, self.dens, nearsing.UPSAMPLE)
        self.check = self.near if up == nearsing.UPSAMPLE else _Grid(drop, self.dens, up)
        self.h = nearsing.spacing(drop)
        self.phi = surface_potential(drop, self.dens) if kind == "ladl" else None

    def upsampled(self, x, n0=None):
        """The near rule of oracle.nearsing (four times upsampled grid) at points x (3, K)."""
        return self.near.rule(self.kind, x, n0)


def lagrange_at(ts, vals, t):
    """The polynomial through (ts[k], vals[k]) at t (Lagrange form); vals (K,) or (K, c)."""
    ts = np.asarray(ts, dtype=np.float64)
    out = 0.0
    for k in range(ts.size):
        w = 1.0
        for l in range(ts.size):
            if l != k:
                w *= (t - ts[l]) / (ts[k] - ts[l])
        out = out + w * vals[k]
    return out


def value(src, x0, n0=None, switch=None, t1=None, dt=None, m=None):
    """Drop j's layer potential at x0 (outside S_j): the upsampled rule at d >= switch h_j, otherwise
    the interpolation through the exterior limit at the closest point and m check points along its
    normal (the module's parameters unless given). Returns (value, d / h_j)."""
    switch = SWITCH if switch is None else switch
    t1, dt, m = (T1 if t1 is None else t1), (DT if dt is None else dt), (M if m is None else m)
    x0 = np.asarray(x0, dtype=np.float64).ravel()
    th, ph, xs, ns, d = closest_point(src.drop, x0, src.near)
    if d < 0.0:
        raise ValueError("target inside the source drop")
    if d >= switch * src.h:
        v = src.upsampled(x0[:, None], n0)
        return (float(v[0]) if v.ndim == 1 else v[:, 0]), d / src.h
    ts = np.concatenate([[0.0], (t1 + dt * np.arange(m)) * src.h])
    chk = src.check.rule(src.kind, xs[:, None] + ts[None, 1:] * ns[:, None], n0)
    lim = exterior_limit(src.drop, src.kind, src.dens, th, ph, n0=n0, phi_coef=src.phi)
    vals = np.concatenate([[lim], chk]) if chk.ndim == 1 else np.concatenate([np.asarray(lim)[:, None], chk], axis=1).T
    return lagrange_at(ts, vals, d), d / src.h
