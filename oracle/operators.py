"""Multi-drop layer operators and their Galerkin systems, plain FP64 numpy (test infrastructure only).

Targets of drop i are the nodes of its degree-p grid; sources of drop j are the nodes of its
degree q = 2p+1 grid (upsampled rule, Section 2.1). For a target on drop i the value is
    sum over j != i of the regular rule (Eq. reg_quadrature) on drop j
  + the singular self-integration on drop i (Eq. mod_weights, rotated pole).
Galerkin coefficients are the forward transform of the target values on drop i's degree-p
grid (inner products (., Y_nm) of Section 2).

Systems (readings of the paper's sign conventions are listed in the design notes):
  electric (Eq. galerkin_En):  1/2 E_n - (R-1)/(R+1) sum_j L_j[E_n] = R/(R+1) E_inf . n
  Stokes   (Eq. main_eq):      (lam_i+1) u - sum_j (lam_j-1) D_j[u] = -sum_j S_j[f/Ca_E - f^E]
"""
from __future__ import annotations

import math

import numpy as np

from . import geometry, quadrature, sh


class DropGeom:
    """Geometry of one drop on its target (degree p) and source (degree q) grids."""

    def __init__(self, xcoef, p: int, lam: float = 1.0, q: int | None = None):
        self.p = p
        self.q = 2 * p + 1 if q is None else q
        self.xcoef = np.asarray(xcoef, dtype=np.float64)
        self.lam = lam
        self.th, self.ph = sh.grid_points(p)
        self.x0, self.n0, self.J0 = geometry.surface_on_grid(self.xcoef, p, p)
        self.xs, self.ns, self.Js = geometry.surface_on_grid(self.xcoef, p, self.q)
        self.ws = sh.grid_weights(self.q) * self.Js
        self._rows = {}

    @property
    def nt(self):
        return self.x0.shape[1]

    def rows(self, kind: str, targets=None):
        """Singular self rows of one kernel for the given target indices (all when None).
        All four kernels are computed together per target and cached."""
        tsel = range(self.nt) if targets is None else targets
        missing = [t for t in tsel if (t, kind) not in self._rows]
        for t in missing:
            r = quadrature.self_rows(self.xcoef, self.p, self.q, self.th[t], self.ph[t],
                                     ["lsl", "ladl", "sto_s", "sto_d"])
            for k, v in r.items():
                self._rows[(t, k)] = v
        return np.stack([self._rows[(t, kind)] for t in tsel])


class System:
    def __init__(self, drops, near: bool = False):
        """near=True applies the nearly-singular correction of oracle.nearsing (drop j's
        contribution at targets near S_j from the upsampled rule)."""
        self.drops = drops
        self.near = near
        self._pairs = None

    def near_pairs(self):
        from . import nearsing
        if self._pairs is None:
            self._pairs = nearsing.near_pairs(self)
        return self._pairs

    # ---------------------------------------------------------------- Laplace
    def laplace_targets(self, kind: str, sigma, i: int, targets=None):
        """Values of sum_j K_j[sigma_j] at targets of drop i (kind 'lsl' or 'ladl')."""
        di = self.drops[i]
        tsel = np.arange(di.nt) if targets is None else np.asarray(targets)
        x0 = di.x0[:, tsel]
        n0 = di.n0[:, tsel]
        out = np.zeros(len(tsel))
        for j, dj in enumerate(self.drops):
            if j == i:
                continue
            dens = sh.sht_inverse(sigma[j], dj.p, dj.q)
            out += quadrature.regular_scalar(kind, x0, n0, dj.xs, dj.ws, dens)
        rows = di.rows(kind, None if targets is None else tsel)
        out += rows @ sigma[i]
        return out

    def laplace_grid(self, kind: str, sigma):
        if self.near:
            from . import nearsing
            return nearsing.corrected_laplace_grid(self, kind, sigma, self.near_pairs())
        return [self.laplace_targets(kind, sigma, i) for i in range(len(self.drops))]

    def laplace_coef(self, kind: str, sigma):
        return [sh.sht_forward(v, d.p, d.p) for v, d in zip(self.laplace_grid(kind, sigma), self.drops)]

    # ---------------------------------------------------------------- Stokes
    def stokes_targets(self, f, u, i: int, targets=None):
        """sum_j S_j[f_j] + sum_j (lam_j - 1) D_j[u_j] at targets of drop i; f,u lists of (3,ncoef)
        (either may be None)."""
        di = self.drops[i]
        tsel = np.arange(di.nt) if targets is None else np.asarray(targets)
        x0 = di.x0[:, tsel]
        out = np.zeros((3, len(tsel)))
        for j, dj in enumerate(self.drops):
            if f is not None:
                if j != i:
                    dens = sh.sht_inverse(f[j], dj.p, dj.q)
                    out += quadrature.regular_tensor("sto_s", x0, dj.xs, dj.ns, dj.ws, dens)
                else:
                    rows = di.rows("sto_s", None if targets is None else tsel)
                    out += np.einsum("tikc,kc->it", rows, f[i])
            if u is not None and dj.lam != 1.0:
                if j != i:
                    dens = sh.sht_inverse(u[j], dj.p, dj.q)
                    out += (dj.lam - 1.0) * quadrature.regular_tensor("sto_d", x0, dj.xs, dj.ns,
                                                                      dj.ws, dens)
                else:
                    rows = di.rows("sto_d", None if targets is None else tsel)
                    out += (dj.lam - 1.0) * np.einsum("tikc,kc->it", rows, u[i])
        return out

    def stokes_grid(self, f, u):
        if self.near:
            from . import nearsing
            return nearsing.corrected_stokes_grid(self, f, u, self.near_pairs())
        return [self.stokes_targets(f, u, i) for i in range(len(self.drops))]

    def stokes_coef(self, f, u):
        return [sh.sht_forward(v, d.p, d.p) for v, d in zip(self.stokes_grid(f, u), self.drops)]

    # ---------------------------------------------------------------- systems
    def pack(self, parts):
        return np.concatenate([np.asarray(a).ravel() for a in parts])

    def unpack(self, vec, ncomp: int):
        out, o = [], 0
        for d in self.drops:
            k = ncomp * sh.ncoef(d.p)
            a = vec[o:o + k]
            out.append(a.reshape(ncomp, -1) if ncomp > 1 else a)
            o += k
        return out

    def electric_matvec(self, R: float, vec):
        """Galerkin form of Eq. galerkin_En: 1/2 sigma - (R-1)/(R+1) sum_j (L_j[sigma], Y)."""
        sig = self.unpack(vec, 1)
        L = self.laplace_coef("ladl", sig)
        return self.pack([0.5 * s - (R - 1.0) / (R + 1.0) * l for s, l in zip(sig, L)])

    def electric_rhs(self, R: float, E_u):
        """R/(R+1) (E_inf . n, Y) for a uniform field E_inf = E_u."""
        E_u = np.asarray(E_u, dtype=np.float64)
        return self.pack([sh.sht_forward(R / (R + 1.0) * (E_u[:, None] * d.n0).sum(axis=0), d.p, d.p)
                          for d in self.drops])

    def stokes_matvec(self, vec):
        """(lam_i + 1) u_i - sum_j (lam_j - 1) (D_j[u_j], Y)."""
        u = self.unpack(vec, 3)
        D = self.stokes_coef(None, u)
        return self.pack([(d.lam + 1.0) * ui - di for ui, di, d in zip(u, D, self.drops)])
