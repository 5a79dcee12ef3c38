"""The Stokes system's self part on the unit sphere and the preconditioner built on it (pins of the oracle
and of the reading behind the library's right preconditioner of the Stokes system).

The self part of the Stokes system of a drop of viscosity ratio lambda (Eq. main_eq in Galerkin form) is
(lambda + 1) u - (lambda - 1) D[u]. On any closed surface the double layer reproduces rigid motions
(D[c] = c, D[omega x x] = omega x x: the stresslet identity of Section 1), so those six modes have the
eigenvalue 2; on the unit sphere the normal field n is an eigenfunction of D with eigenvalue -1 (the
double layer of a uniform expansion), i.e. the eigenvalue 2 lambda. All other eigenvalues mu of D on the
sphere lie in [-1/5, 3/5], so the self part's spectrum clusters near lambda + 1 apart from those seven
modes, which the preconditioner maps to 1. The whole spectrum of both layers on the sphere follows in
closed form from Lamb's solution (the last test), which pins the single and double layer on densities of
every degree, tangential and normal.
"""
import math

import numpy as np
import pytest

import inputs
from oracle import gmres, operators, sh


def _self_matrix(drop):
    sysm = operators.System([drop], near=False)
    n3 = 3 * sh.ncoef(drop.p)
    M = np.zeros((n3, n3))
    for k in range(n3):
        e = np.zeros(n3)
        e[k] = 1.0
        M[:, k] = sysm.stokes_matvec(e)
    return M


def _modes(xcoef, p):
    """Translations (sqrt(4 pi) on Y_00), rotations e_k x x, and the parameter sphere's radial field."""
    nc = sh.ncoef(p)
    xc = np.asarray(xcoef).reshape(3, nc)
    rigid = []
    for k in range(3):
        v = np.zeros((3, nc))
        v[k, 0] = math.sqrt(4 * math.pi)
        rigid.append(v.ravel())
    for k in range(3):
        k1, k2 = (k + 1) % 3, (k + 2) % 3
        v = np.zeros((3, nc))
        v[k1] = -xc[k2]
        v[k2] = xc[k1]
        rigid.append(v.ravel())
    radial = inputs.sphere_coef(p).ravel()
    return np.array(rigid), radial


@pytest.mark.parametrize("lam", [0.3, 4.0])
def test_rigid_and_normal_modes_of_the_sphere(lam):
    p = 5
    drop = operators.DropGeom(inputs.sphere_coef(p), p, lam)
    M = _self_matrix(drop)
    rigid, radial = _modes(drop.xcoef, p)
    for v in rigid:
        np.testing.assert_allclose(M @ v, 2.0 * v, atol=1e-10 * np.abs(v).max())
    np.testing.assert_allclose(M @ radial, 2.0 * lam * radial, atol=1e-10 * np.abs(radial).max())
    # every other eigenvalue (lambda + 1) - (lambda - 1) mu has mu in [-1/5, 3/5]
    ev = np.sort(np.linalg.eigvals(M).real)
    mu = np.sort(((lam + 1.0) - ev) / (lam - 1.0))
    rest = mu[1:-6]
    assert abs(mu[0] + 1.0) < 1e-9 and np.all(np.abs(mu[-6:] - 1.0) < 1e-9)
    assert rest.min() > -0.2 - 1e-9 and rest.max() < 0.6 + 1e-9


def _preconditioner(drops):
    """P^-1 of the library's Stokes preconditioner, per drop: v/(lam+1) + (1/2 - 1/(lam+1)) Q Q^T v
    + (1/(2 lam) - 1/(lam+1)) r r^T v, Q orthonormal over the rigid modes, r the radial field
    orthogonalised against them and normalised."""
    blocks = []
    for d in drops:
        rigid, radial = _modes(d.xcoef, d.p)
        Q, _ = np.linalg.qr(rigid.T)
        r = radial - Q @ (Q.T @ radial)
        r /= np.linalg.norm(r)
        a = 1.0 / (d.lam + 1.0)
        blocks.append((Q, r, a, 0.5 - a, 0.5 / d.lam - a))

    def apply(v):
        out = np.empty_like(v)
        o = 0
        for d, (Q, r, a, cq, cr) in zip(drops, blocks):
            n3 = 3 * sh.ncoef(d.p)
            vi = v[o:o + n3]
            out[o:o + n3] = a * vi + cq * (Q @ (Q.T @ vi)) + cr * r * (r @ vi)
            o += n3
        return out
    return apply


def test_preconditioned_self_part_of_a_sphere_is_identity_on_the_seven_modes():
    p, lam = 5, 7.0
    drop = operators.DropGeom(inputs.sphere_coef(p), p, lam)
    M = _self_matrix(drop)
    Pinv = _preconditioner([drop])
    rigid, radial = _modes(drop.xcoef, p)
    for v in list(rigid) + [radial]:
        np.testing.assert_allclose(M @ Pinv(v), v, atol=1e-10 * np.abs(v).max())
    # the preconditioned spectrum: 1 on the seven modes, (lam+1 - (lam-1) mu)/(lam+1) elsewhere
    n3 = M.shape[0]
    MP = np.column_stack([M @ Pinv(e) for e in np.eye(n3)])
    ev = np.linalg.eigvals(MP).real
    lo = (lam + 1.0 - (lam - 1.0) * 0.6) / (lam + 1.0)
    hi = (lam + 1.0 + (lam - 1.0) * 0.2) / (lam + 1.0)
    assert ev.min() > lo - 1e-9 and ev.max() < hi + 1e-9


def test_preconditioner_cuts_gmres_steps_on_perturbed_drops():
    """Six perturbed drops of viscosity ratios U(0.5, 10): right-preconditioned GMRES reaches the same
    solution in at most three quarters of the plain GMRES steps (plain FP64 oracle GMRES to 1e-10)."""
    rng = np.random.default_rng(3)
    p, centres = 4, []
    while len(centres) < 6:
        c = rng.uniform(-2.6, 2.6, 3)
        if all(np.linalg.norm(c - d) > 2.35 for d in centres):
            centres.append(c)
    drops = [operators.DropGeom(inputs.perturbed_coef(p, rng, 1.0, c), p, float(rng.uniform(0.5, 10.0)))
             for c in centres]
    sysm = operators.System(drops, near=False)
    b = np.concatenate([inputs.random_density(p, rng, 3).ravel() for _ in drops])
    x, info = gmres.gmres(sysm.stokes_matvec, b, tol=1e-10)
    Pinv = _preconditioner(drops)
    y, info_p = gmres.gmres(lambda v: sysm.stokes_matvec(Pinv(v)), b, tol=1e-10)
    xp = Pinv(y)
    assert np.linalg.norm(xp - x) < 1e-8 * np.linalg.norm(x)
    assert info_p["iters"] <= 0.75 * info["iters"], (info_p["iters"], info["iters"])


def _vector_harmonics(p, n, m):
    """Cartesian coefficient arrays (3, ncoef) of Y r_hat, grad_S Y and r_hat x grad_S Y on the unit sphere
    for the real harmonic Y = S_nm (each component has degree <= n + 1 <= p)."""
    th, ph = sh.grid_points(p)
    S, St, Sp = sh.basis(p, np.cos(th), np.sin(th), ph, derivs=True)
    k = sh.idx(n, m)
    rh = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    thh = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)])
    phh = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)])
    fields = (S[k] * rh, St[k] * thh + Sp[k] * phh, St[k] * phh - Sp[k] * thh)
    return [np.stack([sh.sht_forward(f[i], p, p) for i in range(3)]) for f in fields]


@pytest.mark.parametrize("n,m", [(1, 1), (2, 0), (3, -2), (4, 3), (5, 0)])
def test_stokes_operators_on_vector_harmonics_of_the_sphere(n, m):
    """Closed forms on the unit sphere from Lamb's general solution (interior r^n and exterior r^-(n+1)
    pressure harmonics with their potential flows), with the single layer continuous and its traction
    jumping by the density (S[c] = (4/3) c fixes the factor) and the double layer jumping by 2u with
    continuous traction (D[c] = 2c, c, 0 inside, on, outside). With den = (2n-1)(2n+1)(2n+3):
      S[a Y r + b grad Y]: radial 2n(n+1)(2a + 3b)/den, tangential 2(3a + (2n(n+1) + 3) b)/den;
      D[a Y r + b grad Y]: radial 3(a + 2n(n+1) b)/den, tangential 3(2a + 3b)/den;
      S[r x grad Y] = 2/(2n+1), D[r x grad Y] = 3/(2n+1) times the field.
    D's eigenvalues on the poloidal pair are 3/((2n-1)(2n+1)) and -3/((2n+1)(2n+3))."""
    p, lam = 6, 3.0
    drop = operators.DropGeom(inputs.sphere_coef(p), p, lam)
    sysm = operators.System([drop], near=False)
    Yr, Gy, Tor = _vector_harmonics(p, n, m)
    S = lambda v: sysm.stokes_coef([v], None)[0]
    D = lambda v: sysm.stokes_coef(None, [v])[0] / (lam - 1.0)
    den = (2 * n - 1) * (2 * n + 1) * (2 * n + 3)
    nn = n * (n + 1)
    tol = 1e-13
    np.testing.assert_allclose(S(Yr), 2 * nn * 2 / den * Yr + 2 * 3 / den * Gy, atol=tol)
    np.testing.assert_allclose(S(Gy), 2 * nn * 3 / den * Yr + 2 * (2 * nn + 3) / den * Gy, atol=tol)
    np.testing.assert_allclose(D(Yr), 3 / den * Yr + 6 / den * Gy, atol=tol)
    np.testing.assert_allclose(D(Gy), 6 * nn / den * Yr + 9 / den * Gy, atol=tol)
    np.testing.assert_allclose(S(Tor), 2 / (2 * n + 1) * Tor, atol=tol)
    np.testing.assert_allclose(D(Tor), 3 / (2 * n + 1) * Tor, atol=tol)
