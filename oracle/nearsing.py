"""Nearly-singular correction, plain FP64 numpy (test infrastructure only).

Section 2.1 (last paragraph) treats targets close to another drop's surface with the regular
rule on an upsampled grid ("with a reasonable upsampling rate") for points far enough from the
surface, combined with the on-surface rule and 1D interpolation for the closest ones. The paper
gives no parameters; the reading used here:
  * h_j = sqrt(area_j / N_s) is the spacing of drop j's degree-q source grid (q = 2p+1);
  * a target x0 of drop i is near S_j when its distance to the nearest source node of S_j is
    below 6 h_j (beyond that the degree-q rule is accurate to ~1e-11 relative);
  * for near targets, drop j's contribution is the regular rule (Eq. reg_quadrature) on drop
    j's grid upsampled four times in each direction, degree q_n = 4(q+1) - 1. Against closed forms
    on the unit sphere its error at d = h_j is ~1e-11 (single layer), ~1e-9 (field, Stokeslet) and
    ~2e-7 (stresslet of a constant density), at 1.5 h_j 1e-14 to 4e-11, from 2 h_j on rounding.
The interpolation step of the paper, for targets closer than about h_j, is oracle.nearinterp; the
library applies this rule at every near target, and the workloads here keep targets at least
2.6 h_j from other drops (drops 0.1 apart at p = 32), so this module is the library's reference.
"""
from __future__ import annotations

import math

import numpy as np

from . import geometry, quadrature, sh

NEAR_FACTOR = 6.0
UPSAMPLE = 4


def spacing(drop) -> float:
    area = float(drop.ws.sum())
    return math.sqrt(area / drop.xs.shape[1])


def near_degree(drop) -> int:
    return UPSAMPLE * (drop.q + 1) - 1


def near_pairs(system):
    """All (i, t, j): target t of drop i within NEAR_FACTOR h_j of a source node of drop j."""
    out = []
    for i, di in enumerate(system.drops):
        for j, dj in enumerate(system.drops):
            if i == j:
                continue
            lim = NEAR_FACTOR * spacing(dj)
            for t in range(di.nt):
                d = dj.xs - di.x0[:, t:t + 1]
                if math.sqrt((d * d).sum(axis=0).min()) < lim:
                    out.append((i, t, j))
    return out


def near_pairs_of(system, i: int, targets=None):
    """The near pairs (i, t, j) of drop i's targets (all of them, or the given ones), by the same rule as
    near_pairs; drops j whose bounding sphere (centre, largest node distance) is farther than
    NEAR_FACTOR h_j from every target of drop i are skipped without testing their nodes."""
    di = system.drops[i]
    ts = np.arange(di.nt) if targets is None else np.asarray(targets, dtype=int)
    x0 = di.x0[:, ts]
    out = []
    for j, dj in enumerate(system.drops):
        if j == i:
            continue
        lim = NEAR_FACTOR * spacing(dj)
        c = dj.xs.mean(axis=1)
        rad = math.sqrt(((dj.xs - c[:, None]) ** 2).sum(axis=0).max())
        dc = np.sqrt(((x0 - c[:, None]) ** 2).sum(axis=0))
        cand = np.nonzero(dc < rad + lim)[0]
        for k in cand:
            d = dj.xs - x0[:, k:k + 1]
            if math.sqrt((d * d).sum(axis=0).min()) < lim:
                out.append((i, int(ts[k]), j))
    return out


class _Fine:
    def __init__(self, dj):
        self.q = near_degree(dj)
        self.x, self.n, J = geometry.surface_on_grid(dj.xcoef, dj.p, self.q)
        self.w = sh.grid_weights(self.q) * J


def _near_by_target(system, i, targets, pairs):
    """{position in targets: [source drops j]} of the near pairs whose target lies in drop i's list."""
    pos = {int(t): k for k, t in enumerate(targets)}
    out = {}
    for (ii, t, j) in (near_pairs(system) if pairs is None else pairs):
        if ii == i and t in pos:
            out.setdefault(pos[t], []).append(j)
    return out


def corrected_laplace_targets(system, kind: str, sigma, i: int, targets, pairs=None, fine=None):
    """Values of sum_j K_j[sigma_j] at the given targets of drop i, drop j's contribution at targets
    near S_j taken from the upsampled rule (fine: optional cache {j: _Fine})."""
    targets = np.asarray(targets)
    out = system.laplace_targets(kind, sigma, i, targets)
    fine = {} if fine is None else fine
    di = system.drops[i]
    for k, js in _near_by_target(system, i, targets, pairs).items():
        t = int(targets[k])
        x0, n0 = di.x0[:, t:t + 1], di.n0[:, t:t + 1]
        for j in js:
            dj = system.drops[j]
            if j not in fine:
                fine[j] = _Fine(dj)
            F = fine[j]
            reg = quadrature.regular_scalar(kind, x0, n0, dj.xs, dj.ws, sh.sht_inverse(sigma[j], dj.p, dj.q))[0]
            up = quadrature.regular_scalar(kind, x0, n0, F.x, F.w, sh.sht_inverse(sigma[j], dj.p, F.q))[0]
            out[k] += up - reg
    return out


def corrected_stokes_targets(system, f, u, i: int, targets, pairs=None, fine=None):
    """sum_j S_j[f_j] + (lam_j - 1) D_j[u_j] at the given targets of drop i, with the upsampled rule
    at near targets."""
    targets = np.asarray(targets)
    out = system.stokes_targets(f, u, i, targets)
    fine = {} if fine is None else fine
    di = system.drops[i]
    for k, js in _near_by_target(system, i, targets, pairs).items():
        t = int(targets[k])
        x0 = di.x0[:, t:t + 1]
        for j in js:
            dj = system.drops[j]
            if j not in fine:
                fine[j] = _Fine(dj)
            F = fine[j]
            if f is not None:
                out[:, k] += quadrature.regular_tensor("sto_s", x0, F.x, F.n, F.w, sh.sht_inverse(f[j], dj.p, F.q))[:, 0]
                out[:, k] -= quadrature.regular_tensor("sto_s", x0, dj.xs, dj.ns, dj.ws,
                                                       sh.sht_inverse(f[j], dj.p, dj.q))[:, 0]
            if u is not None and dj.lam != 1.0:
                out[:, k] += (dj.lam - 1.0) * quadrature.regular_tensor("sto_d", x0, F.x, F.n, F.w,
                                                                        sh.sht_inverse(u[j], dj.p, F.q))[:, 0]
                out[:, k] -= (dj.lam - 1.0) * quadrature.regular_tensor("sto_d", x0, dj.xs, dj.ns, dj.ws,
                                                                        sh.sht_inverse(u[j], dj.p, dj.q))[:, 0]
    return out


def corrected_laplace_grid(system, kind: str, sigma, pairs=None):
    """Target values of sum_j K_j[sigma_j] with drop j's contribution at near targets taken
    from the upsampled rule."""
    out = [system.laplace_targets(kind, sigma, i) for i in range(len(system.drops))]
    pairs = near_pairs(system) if pairs is None else pairs
    fine, dens = {}, {}
    for (i, t, j) in pairs:
        di, dj = system.drops[i], system.drops[j]
        if j not in fine:
            fine[j] = _Fine(dj)
            dens[j] = (sh.sht_inverse(sigma[j], dj.p, dj.q), sh.sht_inverse(sigma[j], dj.p, fine[j].q))
        F = fine[j]
        x0, n0 = di.x0[:, t:t + 1], di.n0[:, t:t + 1]
        reg = quadrature.regular_scalar(kind, x0, n0, dj.xs, dj.ws, dens[j][0])[0]
        up = quadrature.regular_scalar(kind, x0, n0, F.x, F.w, dens[j][1])[0]
        out[i][t] += up - reg
    return out


def corrected_stokes_grid(system, f, u, pairs=None):
    """sum_j S_j[f_j] + (lam_j - 1) D_j[u_j] with the upsampled rule at near targets."""
    out = [system.stokes_targets(f, u, i) for i in range(len(system.drops))]
    pairs = near_pairs(system) if pairs is None else pairs
    fine, dens = {}, {}
    for (i, t, j) in pairs:
        di, dj = system.drops[i], system.drops[j]
        if j not in fine:
            F = fine[j] = _Fine(dj)
            dens[j] = [None if a is None else (sh.sht_inverse(a[j], dj.p, dj.q), sh.sht_inverse(a[j], dj.p, F.q))
                       for a in (f, u)]
        F = fine[j]
        fd, ud = dens[j]
        x0 = di.x0[:, t:t + 1]
        corr = np.zeros(3)
        if fd is not None:
            corr += quadrature.regular_tensor("sto_s", x0, F.x, F.n, F.w, fd[1])[:, 0]
            corr -= quadrature.regular_tensor("sto_s", x0, dj.xs, dj.ns, dj.ws, fd[0])[:, 0]
        if ud is not None and dj.lam != 1.0:
            corr += (dj.lam - 1.0) * quadrature.regular_tensor("sto_d", x0, F.x, F.n, F.w, ud[1])[:, 0]
            corr -= (dj.lam - 1.0) * quadrature.regular_tensor("sto_d", x0, dj.xs, dj.ns, dj.ws, ud[0])[:, 0]
        out[i][:, t] += corr
    return out
