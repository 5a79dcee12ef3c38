"""Forces, surfactant rates and the time step, plain FP64 numpy (test infrastructure only).

Follows Section 1 (steps i-viii) and Algorithm 1 of the paper:
  * E_n from the Galerkin electric system (Eq. galerkin_En); the charge q = (1 - 1/R) E_n
    (jump of E_n with Eq. EneEni) and its single-layer potential phi_q = S_L[q] (Eq. BIE01
    as a potential); the tangential mean field E_t = -grad_S (phi_inf + phi_q) (Eq. E_t).
  * electric traction (Eq. el_force) with eps = 1 in the non-dimensional units;
  * Langmuir tension normalised to gamma(1) = 1 (Eq. langmuir), interfacial force
    f = 2 gamma H n - grad_S gamma (Eq. interfacial_force), H = 1/2 div_S n (= 1 on the unit
    sphere);
  * Stokes solve with right-hand side -sum_j S_j[f/Ca_E - f^E] (Eq. main_eq);
  * surfactant rate for nodes that move with the full velocity (Eq. surfactant0 written in
    material form, Pe = infinity): dGamma/dt = -Gamma div_S u;
  * midpoint rule for x and the explicit stage of the IMEX scheme for Gamma (Algorithm 1);
    error estimate = grid max-norm difference between the midpoint step and the explicit
    Euler step of x and Gamma.
Nonlinear products are evaluated on each drop's degree 2p+1 grid and projected back to degree
p (Galerkin inner products), i.e. de-aliased.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import geometry, gmres, operators, sh


def basis2(p: int, theta, phi):
    """Real basis with first and second derivatives in (theta, phi) at points away from the
    poles: returns S, S_t, S_p, S_tt, S_tp, S_pp (phi derivatives NOT divided by sin).
    Second theta derivative from the associated Legendre equation
    P'' = -cot(t) P' - (n(n+1) - m^2/sin^2 t) P."""
    theta = np.asarray(theta, dtype=np.float64).ravel()
    phi = np.asarray(phi, dtype=np.float64).ravel()
    ct, st = np.cos(theta), np.sin(theta)
    S, St, Sps = sh.basis(p, ct, st, phi, derivs=True)
    Sp = Sps * st
    Stt = np.zeros_like(S)
    Stp = np.zeros_like(S)
    Spp = np.zeros_like(S)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            i = sh.idx(n, m)
            am = abs(m)
            Stt[i] = -(ct / st) * St[i] - (n * (n + 1) - am * am / (st * st)) * S[i]
            Spp[i] = -am * am * S[i]
            if m > 0:
                Stp[i] = -m * St[sh.idx(n, -m)]
            elif m < 0:
                Stp[i] = am * St[sh.idx(n, am)]
    return S, St, Sp, Stt, Stp, Spp


class SurfaceGrid:
    """Geometry of one drop on a Gaussian grid of degree q (no pole nodes)."""

    def __init__(self, xcoef, p: int, q: int):
        self.p, self.q = p, q
        th, ph = sh.grid_points(q)
        self.theta, self.phi = th, ph
        B = basis2(p, th, ph)
        self.B = B
        self._xcoef = np.asarray(xcoef)
        x, xt, xp, xtt, xtp, xpp = (np.asarray(xcoef) @ b for b in B)
        c = np.cross(xt.T, xp.T).T
        W = np.sqrt((c * c).sum(axis=0))
        self.x, self.xt, self.xp = x, xt, xp
        self.n = c / W
        self.J = W / np.sin(th)
        E = (xt * xt).sum(axis=0)
        F = (xt * xp).sum(axis=0)
        G = (xp * xp).sum(axis=0)
        L = (xtt * self.n).sum(axis=0)
        M = (xtp * self.n).sum(axis=0)
        N = (xpp * self.n).sum(axis=0)
        self.E, self.F, self.G = E, F, G
        self.det = E * G - F * F
        self.H = -(E * N - 2.0 * F * M + G * L) / (2.0 * self.det)
        self.omega = sh.grid_weights(q)

    def values(self, coef):
        return np.asarray(coef) @ self.B[0]

    def grad(self, coef):
        """Surface gradient of a scalar degree-p expansion: (3, npts)."""
        ft = np.asarray(coef) @ self.B[1]
        fp = np.asarray(coef) @ self.B[2]
        a = (self.G * ft - self.F * fp) / self.det
        b = (self.E * fp - self.F * ft) / self.det
        return a * self.xt + b * self.xp

    def div(self, vcoef):
        """Surface divergence of a vector field given by 3 degree-p expansions."""
        ut = np.asarray(vcoef) @ self.B[1]
        up = np.asarray(vcoef) @ self.B[2]
        a = (ut * self.xt).sum(axis=0)
        b = (ut * self.xp).sum(axis=0)
        c = (up * self.xt).sum(axis=0)
        d = (up * self.xp).sum(axis=0)
        return (self.G * a - self.F * (b + c) + self.E * d) / self.det

    def project(self, vals):
        """Galerkin projection onto degree p by the regular rule of this grid."""
        return (np.asarray(vals) * self.omega) @ self.B[0].T

    def laplace_beltrami(self, coef):
        """Surface Laplacian of a scalar degree-p expansion in the (theta, phi) chart:
        Delta_S f = g^{ab} (f_ab - Gamma^c_ab f_c), Gamma^c_ab = g^{cd} x_d . x_ab."""
        c = np.asarray(coef)
        ft, fp, ftt, ftp, fpp = (c @ self.B[k] for k in (1, 2, 3, 4, 5))
        xc = self._xcoef
        xtt, xtp, xpp = (xc @ self.B[k] for k in (3, 4, 5))
        E, F, G, det = self.E, self.F, self.G, self.det
        gtt, gtp, gpp = G / det, -F / det, E / det          # inverse metric
        def christ(xab):
            a = (self.xt * xab).sum(0)
            b = (self.xp * xab).sum(0)
            return gtt * a + gtp * b, gtp * a + gpp * b      # Gamma^theta_ab, Gamma^phi_ab
        Ttt, Ptt = christ(xtt)
        Ttp, Ptp = christ(xtp)
        Tpp, Ppp = christ(xpp)
        return (gtt * (ftt - Ttt * ft - Ptt * fp) + 2.0 * gtp * (ftp - Ttp * ft - Ptp * fp)
                + gpp * (fpp - Tpp * ft - Ppp * fp))


@dataclass
class Params:
    R: float = 2.0
    Q: float = 0.5
    Ca_E: float = 0.1
    beta: float = 0.2
    x_s: float = 0.5
    E_u: tuple = (0.0, 0.0, 1.0)
    E_q: float = 0.0            # strength of the linear field E_q G x added to the uniform one
    E_G: tuple = ((1.0, 0.0, 0.0), (0.0, -1.0, 0.0), (0.0, 0.0, 0.0))   # its shape G (symmetric,
    # traceless); the quadrupole field of Section 3, phi = -E_q r^2 P_2, is diag(-1, -1, 2)
    gmres_tol: float = 1e-12
    Pe: float = math.inf        # surfactant Peclet number (infinity: no diffusion)
    eos: str = "langmuir"       # equation of state: "langmuir" (beta, x_s) or "linear" (beta as beta_t)


def langmuir(G, beta: float, x_s: float):
    """Eq. langmuir normalised so that gamma(1) = 1; returns gamma and d gamma / d Gamma."""
    den = 1.0 + beta * math.log(1.0 - x_s)
    g = (1.0 + beta * np.log(1.0 - x_s * G)) / den
    dg = (-beta * x_s / (1.0 - x_s * G)) / den
    return g, dg


def linear_tension(G, beta_t: float):
    """The linear equation of state of Section 1, gamma = 1 + beta_t (1 - Gamma) (normalised on the
    equilibrium tension); returns gamma and d gamma / d Gamma."""
    G = np.asarray(G, dtype=np.float64)
    return 1.0 + beta_t * (1.0 - G), np.full_like(G, -beta_t)


def tension(G, prm: "Params"):
    """The tension law the parameters select."""
    if prm.eos == "linear":
        return linear_tension(G, prm.beta)
    if prm.eos != "langmuir":
        raise ValueError("unknown equation of state %r" % prm.eos)
    return langmuir(G, prm.beta, prm.x_s)


def electric_traction(En, Et, n, R: float, Q: float):
    """Eq. el_force: 1/2 [(1 - Q/R^2) E_n^2 - (1 - Q) |E_t|^2] n + (1 - Q/R) E_n E_t."""
    Et2 = (Et * Et).sum(axis=0)
    return 0.5 * ((1.0 - Q / R ** 2) * En ** 2 - (1.0 - Q) * Et2) * n + (1.0 - Q / R) * En * Et


def far_field(x, prm: Params):
    Eu = np.asarray(prm.E_u, dtype=np.float64)[:, None]
    return Eu + prm.E_q * (np.asarray(prm.E_G, dtype=np.float64) @ x)


def rates(xcoefs, gcoefs, ps, lams, prm: Params, info=None, near: bool = True):
    """Velocity and surfactant-rate coefficients of every drop for one geometry
    (steps i-vi of Section 1 and the explicit rate g_E of Algorithm 1); near=True applies the
    nearly-singular correction of oracle.nearsing to every layer operator."""
    drops = [operators.DropGeom(xc, p, lam) for xc, p, lam in zip(xcoefs, ps, lams)]
    sysm = operators.System(drops, near=near)
    R = prm.R
    # (i) E_n: 1/2 E_n - (R-1)/(R+1) L[E_n] = R/(R+1) E_inf . n
    b = sysm.pack([sh.sht_forward(R / (R + 1.0) * (far_field(d.x0, prm) * d.n0).sum(axis=0), d.p, d.p)
                   for d in drops])
    En, ie = gmres.gmres(lambda v: sysm.electric_matvec(R, v), b, tol=prm.gmres_tol)
    Enc = sysm.unpack(En, 1)
    # (ii) potential of the charge q = (1 - 1/R) E_n
    q = [(1.0 - 1.0 / R) * e for e in Enc]
    phi = sysm.laplace_coef("lsl", q)
    # (iii)-(v) tractions on each drop's upsampled grid, projected to degree p
    t_coefs = []
    grids = []
    for d, e, ph, g in zip(drops, Enc, phi, gcoefs):
        sg = SurfaceGrid(d.xcoef, d.p, d.q)
        grids.append(sg)
        Einf = far_field(sg.x, prm)
        Et = (Einf - (Einf * sg.n).sum(axis=0) * sg.n) - sg.grad(ph)
        fE = electric_traction(sg.values(e), Et, sg.n, R, prm.Q)
        Gv = sg.values(g)
        gam, dgam = tension(Gv, prm)
        f = 2.0 * gam * sg.H * sg.n - dgam * sg.grad(g)
        t_coefs.append(sg.project(f / prm.Ca_E - fE))
    # (vi) Stokes: (lam_i+1) u - sum (lam_j-1) D_j[u] = -sum S_j[t]
    bs = -sysm.pack([a.ravel() for a in sysm.stokes_coef(t_coefs, None)])
    u, iu = gmres.gmres(sysm.stokes_matvec, bs, tol=prm.gmres_tol)
    uc = sysm.unpack(u, 3)
    # surfactant rate in material form: -Gamma div_S u
    gE = [sg.project(-sg.values(g) * sg.div(uu)) for sg, g, uu in zip(grids, gcoefs, uc)]
    if info is not None:
        info.update({"En": Enc, "phi": phi, "traction": t_coefs, "iters": (ie["iters"], iu["iters"])})
    return uc, gE


def grid_max_diff(acoefs, bcoefs, ps, ncomp):
    m = 0.0
    for a, b, p in zip(acoefs, bcoefs, ps):
        d = sh.sht_inverse(np.asarray(a) - np.asarray(b), p, p)
        if ncomp > 1:
            m = max(m, float(np.sqrt((d * d).sum(axis=0)).max()))
        else:
            m = max(m, float(np.abs(d).max()))
    return m


def diffusion_solve(xcoef, p: int, rhs, c: float, tol: float = 1e-13):
    """Solve (I - c Delta_S) G = rhs in Galerkin form on the surface xcoef (degree 2p+1 grid),
    by GMRES right-preconditioned with the sphere eigenvalues: M^{-1} = diag(1/(1 + c n(n+1)/a^2)),
    a^2 = area / (4 pi). Returns the coefficients of G."""
    sg = SurfaceGrid(xcoef, p, 2 * p + 1)
    a2 = float((sg.omega * sg.J).sum()) / (4 * math.pi)
    nn = np.array([n for n in range(p + 1) for _ in range(2 * n + 1)], dtype=np.float64)
    minv = 1.0 / (1.0 + c * nn * (nn + 1) / a2)
    A = lambda y: minv * y - c * sg.project(sg.laplace_beltrami(minv * y))
    y, info = gmres.gmres(A, np.asarray(rhs), tol=tol)
    return minv * y


def step(xcoefs, gcoefs, ps, lams, dt: float, prm: Params, near: bool = True):
    """One midpoint step (Algorithm 1). Returns new x, Gamma and the error estimate
    err = max(err_drop, err_surfactant) against explicit Euler. With a finite Peclet number the
    surfactant follows the IMEX scheme of Algorithm 1: the half step is implicit in the
    diffusion on the half-step surface, (I - dt/(2 Pe) Delta_S) G_half = G + dt/2 g_E, and the full
    step adds dt (g_E + Delta_S G_half / Pe) evaluated at the half step."""
    u0, g0 = rates(xcoefs, gcoefs, ps, lams, prm, near=near)
    xh = [x + 0.5 * dt * u for x, u in zip(xcoefs, u0)]
    gh = [g + 0.5 * dt * r for g, r in zip(gcoefs, g0)]
    if math.isfinite(prm.Pe):
        gh = [diffusion_solve(x, p, g, 0.5 * dt / prm.Pe) for x, p, g in zip(xh, ps, gh)]
    u1, g1 = rates(xh, gh, ps, lams, prm, near=near)
    if math.isfinite(prm.Pe):
        g1 = [r + SurfaceGrid(x, p, 2 * p + 1).project(
            SurfaceGrid(x, p, 2 * p + 1).laplace_beltrami(g)) / prm.Pe for r, x, p, g in zip(g1, xh, ps, gh)]
    xn = [x + dt * u for x, u in zip(xcoefs, u1)]
    gn = [g + dt * r for g, r in zip(gcoefs, g1)]
    xe = [x + dt * u for x, u in zip(xcoefs, u0)]
    ge = [g + dt * r for g, r in zip(gcoefs, g0)]
    err = max(grid_max_diff(xn, xe, ps, 3), grid_max_diff(gn, ge, ps, 1))
    return xn, gn, err, {"u0": u0, "u1": u1, "g0": g0, "g1": g1}


def surfactant_mass(xcoef, gcoef, p: int, q: int | None = None) -> float:
    q = 2 * p + 1 if q is None else q
    sg = SurfaceGrid(xcoef, p, q)
    return float((sg.omega * sg.J * sg.values(gcoef)).sum())
