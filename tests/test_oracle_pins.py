"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics (CPU only).

Each test names what it pins. Together they are chosen so that a dropped term, a wrong sign,
a wrong index or a transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy.special import sph_harm_y

import inputs
from oracle import geometry, gmres, operators, physics, quadrature, sh


# --------------------------------------------------------------------------- basis / SHT

def test_basis_and_derivatives_match_library_harmonics():
    """Eq. normalized_spharm (with the Condon-Shortley phase of Eq. pneg): the real basis and
    its theta / phi derivatives equal sqrt(2) Re/Im of scipy's complex harmonics."""
    rng = np.random.default_rng(0)
    th = rng.uniform(0.0, np.pi, 40)
    ph = rng.uniform(0.0, 2 * np.pi, 40)
    p = 11
    S, St, Sp = sh.basis(p, np.cos(th), np.sin(th), ph, derivs=True)
    for n in range(p + 1):
        for m in range(0, n + 1):
            Y, dY = sph_harm_y(n, m, th, ph, diff_n=1)
            f = 1.0 if m == 0 else math.sqrt(2.0)
            np.testing.assert_allclose(S[sh.idx(n, m)], f * Y.real, atol=1e-13)
            np.testing.assert_allclose(St[sh.idx(n, m)], f * dY[:, 0].real, atol=1e-12)
            np.testing.assert_allclose(Sp[sh.idx(n, m)], f * dY[:, 1].real / np.sin(th), atol=1e-12)
            if m > 0:
                np.testing.assert_allclose(S[sh.idx(n, -m)], f * Y.imag, atol=1e-13)
                np.testing.assert_allclose(St[sh.idx(n, -m)], f * dY[:, 0].imag, atol=1e-12)
                np.testing.assert_allclose(Sp[sh.idx(n, -m)], f * dY[:, 1].imag / np.sin(th),
                                           atol=1e-12)


def test_derivatives_accurate_near_pole():
    """The division-free derivative identities stay exact where theta -> 0 (finite differences
    in theta at theta = 1e-7 would be useless; compare with the analytic pole limit of Y_11)."""
    th = np.array([1e-9, 1e-7])
    S, St, Sp = sh.basis(3, np.cos(th), np.sin(th), np.zeros(2), derivs=True)
    c = -math.sqrt(3.0 / (4 * math.pi))           # S_11 = c sin(t) cos(f)
    np.testing.assert_allclose(St[sh.idx(1, 1)], c * np.cos(th), rtol=1e-14)
    np.testing.assert_allclose(Sp[sh.idx(1, -1)], c * np.ones(2), rtol=1e-14)


@pytest.mark.parametrize("p,q", [(6, 6), (6, 13), (10, 21)])
def test_sht_roundtrip_and_orthonormality(p, q):
    """Gauss-Legendre in theta and the trapezoid rule in phi (Eq. spharm_ex grid) integrate
    products of degree <= p harmonics exactly: forward(inverse(c)) = c."""
    rng = np.random.default_rng(p + q)
    c = rng.standard_normal((2, sh.ncoef(p)))
    np.testing.assert_allclose(sh.sht_forward(sh.sht_inverse(c, p, q), p, q), c, atol=1e-13)
    G = (sh.grid_basis(p, q) * sh.grid_weights(q)) @ sh.grid_basis(p, q).T
    np.testing.assert_allclose(G, np.eye(sh.ncoef(p)), atol=1e-13)


def test_regular_weights_sum_to_sphere_area():
    """Eq. reg_quadrature read with the trapezoid spacing pi/(q+1): weights sum to 4 pi."""
    for q in (4, 9, 33):
        assert abs(sh.grid_weights(q).sum() - 4 * math.pi) < 1e-12


# --------------------------------------------------------------------------- geometry

def test_unit_sphere_geometry():
    """Unit sphere: J = 1, n = x, area 4 pi, volume 4 pi / 3."""
    p = 5
    x, n, J = geometry.surface_on_grid(inputs.sphere_coef(p), p, 11)
    np.testing.assert_allclose(J, 1.0, atol=1e-14)
    np.testing.assert_allclose(n, x, atol=1e-14)
    np.testing.assert_allclose((x * x).sum(axis=0), 1.0, atol=1e-14)
    assert abs(geometry.area(inputs.sphere_coef(p), p, 11) - 4 * math.pi) < 1e-12
    assert abs(geometry.volume(inputs.sphere_coef(p), p, 11) - 4 * math.pi / 3) < 1e-12


def test_ellipsoid_volume_and_normal():
    """Affine image of the sphere (x, y, z) -> (a x, b y, c z): volume 4 pi a b c / 3 and
    normal parallel to (x/a^2, y/b^2, z/c^2)."""
    p = 4
    a, b, c = 1.3, 0.8, 1.1
    xc = inputs.sphere_coef(p)
    xc[0] *= a
    xc[1] *= b
    xc[2] *= c
    assert abs(geometry.volume(xc, p, 9) - 4 * math.pi * a * b * c / 3) < 1e-12
    x, n, _ = geometry.surface_on_grid(xc, p, 9)
    g = x / np.array([a * a, b * b, c * c])[:, None]
    g /= np.sqrt((g * g).sum(axis=0))
    np.testing.assert_allclose(n, g, atol=1e-13)


# --------------------------------------------------------------------------- quadrature

def test_modified_weights_integrate_inverse_distance():
    """Eq. mod_weights: the rule sum mu F integrates F = g / |N - y| exactly for band-limited
    g; with g = 1 the integral is 4 pi and with g = P_l(cos t) it is 4 pi / (2l+1)."""
    q = 15
    mu = quadrature.modified_weights(q)
    th, _ = sh.grid_points(q)
    inv = 1.0 / (2.0 * np.sin(0.5 * th))
    assert abs((mu * inv).sum() - 4 * math.pi) < 1e-12
    from scipy.special import eval_legendre
    for l in (1, 4, 9, 15):
        got = (mu * eval_legendre(l, np.cos(th)) * inv).sum()
        assert abs(got - 4 * math.pi / (2 * l + 1)) < 1e-12


def test_single_layer_eigenrelation_unit_sphere():
    """(1/4pi) int Y_lm / r dS = Y_lm / (2l+1) on the unit sphere, at every target, exact to
    round-off with the rotated-pole modified weights."""
    p = 7
    rng = np.random.default_rng(1)
    sig = inputs.random_density(p, rng)[0]
    d = operators.DropGeom(inputs.sphere_coef(p), p)
    got = d.rows("lsl") @ sig
    scale = np.array([1.0 / (2 * n + 1) for n in range(p + 1) for _ in range(2 * n + 1)])
    np.testing.assert_allclose(got, sh.sht_inverse(sig * scale, p, p), atol=1e-13)
    # on the sphere (x0 - x).n0 = r^2/2, so the target-normal double layer is half of it
    np.testing.assert_allclose(d.rows("ladl") @ sig, 0.5 * got, atol=1e-13)


def test_stokes_identities_unit_sphere():
    """Unit sphere: S[c] = (4/3) c (translating-sphere traction), D[c] = c (stresslet
    identity with xh = x0 - x, Eq. GandT) and S[n] = 0 (G is divergence free)."""
    p = 6
    d = operators.DropGeom(inputs.sphere_coef(p), p)
    c = np.array([0.3, -0.7, 1.1])
    ccoef = np.zeros((3, sh.ncoef(p)))
    ccoef[:, 0] = c * math.sqrt(4 * math.pi)
    ncoef = inputs.sphere_coef(p)
    S = np.einsum("tikc,kc->it", d.rows("sto_s"), ccoef)
    D = np.einsum("tikc,kc->it", d.rows("sto_d"), ccoef)
    Sn = np.einsum("tikc,kc->it", d.rows("sto_s"), ncoef)
    np.testing.assert_allclose(S, (4.0 / 3.0) * c[:, None] * np.ones_like(S), atol=1e-13)
    np.testing.assert_allclose(D, c[:, None] * np.ones_like(D), atol=1e-13)
    np.testing.assert_allclose(Sn, 0.0, atol=1e-13)


def test_stresslet_identity_perturbed_drop_converges():
    """D[c] = c on any smooth closed surface; on a perturbed drop the rotated-pole rule
    approaches it spectrally as the grid is refined."""
    rng = np.random.default_rng(5)
    errs = []
    c = np.array([0.2, 0.5, -0.4])
    for p in (6, 10):
        xc = inputs.perturbed_coef(p, np.random.default_rng(5), 1.0, (0, 0, 0), lmax=4)
        d = operators.DropGeom(xc, p)
        ccoef = np.zeros((3, sh.ncoef(p)))
        ccoef[:, 0] = c * math.sqrt(4 * math.pi)
        sel = np.arange(0, d.nt, 5)
        D = np.einsum("tikc,kc->it", d.rows("sto_d", sel), ccoef)
        errs.append(np.abs(D - c[:, None]).max())
    assert errs[1] < 1e-5 and errs[1] < errs[0] / 10


def test_target_normal_double_layer_gauss_flux():
    """Eq. E_n uses the normal at the target: integrating L[sigma] over the surface gives
    (1/2) int sigma dS by Gauss' flux theorem. The source-normal double layer would give a
    different value off the sphere, so this fixes the normal's position."""
    p = 8
    xc = inputs.perturbed_coef(p, np.random.default_rng(7), 1.0, (0, 0, 0), lmax=3)
    d = operators.DropGeom(xc, p)
    sig = inputs.random_density(p, np.random.default_rng(8), decay=2.0)[0]
    L = d.rows("ladl") @ sig
    lhs = (sh.grid_weights(p) * d.J0 * L).sum()
    rhs = 0.5 * (d.ws * sh.sht_inverse(sig, p, d.q)).sum()
    assert abs(lhs - rhs) < 1e-6 * abs(rhs)


def test_rotation_spin_changes_result_only_spectrally():
    """The rotated-pole rule does not depend on the spin about the pole beyond its own
    quadrature error (the paper fixes only that the target becomes the north pole)."""
    p = 8
    xc = inputs.perturbed_coef(p, np.random.default_rng(3), 1.0, (0, 0, 0), lmax=3)
    th, ph = sh.grid_points(p)
    sig = inputs.random_density(p, np.random.default_rng(4), decay=2.0)[0]
    for t in (3, 40, 100):
        a = quadrature.self_rows(xc, p, 2 * p + 1, th[t], ph[t], ["ladl"])["ladl"] @ sig
        b = quadrature.self_rows(xc, p, 2 * p + 1, th[t], ph[t], ["ladl"], gamma=0.37)["ladl"] @ sig
        assert abs(a - b) < 1e-6 * (abs(a) + 1e-3)


def test_regular_sums_far_field_identities():
    """Between well-separated drops: the flux of a point source through a closed surface
    that does not contain it is zero, D_j[c] = 0 outside S_j and S_j[n_j] = 0."""
    p = 8
    da = operators.DropGeom(inputs.sphere_coef(p, 1.0, (0, 0, 0)), p)
    db = operators.DropGeom(inputs.perturbed_coef(p, np.random.default_rng(2), 1.0, (0, 0, 4.0),
                                                  lmax=3), p)
    # flux through drop b's surface of the field of drop a's sources
    sig = np.ones(da.xs.shape[1])
    vals = np.array([quadrature.regular_scalar("ladl", db.x0[:, t:t + 1], db.n0[:, t:t + 1],
                                               da.xs, da.ws, sig)[0] for t in range(db.nt)])
    assert abs((sh.grid_weights(p) * db.J0 * vals).sum()) < 1e-9
    c = np.array([0.4, 0.1, -0.9])[:, None] * np.ones(da.xs.shape[1])
    D = quadrature.regular_tensor("sto_d", db.x0, da.xs, da.ns, da.ws, c)
    np.testing.assert_allclose(D, 0.0, atol=1e-12)
    S = quadrature.regular_tensor("sto_s", db.x0, da.xs, da.ns, da.ws, da.ns)
    np.testing.assert_allclose(S, 0.0, atol=1e-12)
    # the single layer of a unit density on a unit sphere is 1/|x0| outside it
    out = quadrature.regular_scalar("lsl", db.x0, db.n0, da.xs, da.ws, sig)
    np.testing.assert_allclose(out, 1.0 / np.sqrt((db.x0 ** 2).sum(axis=0)), rtol=1e-12)


# --------------------------------------------------------------------------- systems

@pytest.mark.parametrize("R", [0.1, 2.0])
def test_electric_solution_unit_sphere(R):
    """Eq. E_n on a unit sphere in a uniform field: E_n = 3R/(R+2) E_inf . n."""
    p = 6
    sysm = operators.System([operators.DropGeom(inputs.sphere_coef(p), p)])
    E = np.array([0.3, 0.0, 1.0])
    x, info = gmres.gmres(lambda v: sysm.electric_matvec(R, v), sysm.electric_rhs(R, E), tol=1e-13)
    En = sh.sht_inverse(x, p, p)
    np.testing.assert_allclose(En, 3 * R / (R + 2) * (E[:, None] * sysm.drops[0].n0).sum(axis=0),
                               atol=1e-13)


@pytest.mark.parametrize("R", [0.1, 2.0])
def test_electric_solution_unit_sphere_linear_field(R):
    """A linear far field E = G x (G symmetric, traceless: the quadrupole (-x, -y, 2z) and (x, -y, 0)) on
    the unit sphere, through the field-shape path of the rates: its normal component is a degree-2
    harmonic, the outer potential -r^2 h/2 + B r^-3 h with interior A r^2 h, and continuity of the potential
    and of the current (R times the interior normal field) give E_n = 5R/(2R+3) E . n (degree l in
    general: (2l+1) R / (l R + l + 1), 3R/(R+2) for the uniform field)."""
    p = 6
    for G in (np.diag([-1.0, -1.0, 2.0]), np.diag([1.0, -1.0, 0.0])):
        prm = physics.Params(R=R, Q=0.5, E_u=(0.0, 0.0, 0.0), E_q=0.7, E_G=tuple(map(tuple, G)),
                             gmres_tol=1e-13)
        info = {}
        physics.rates([inputs.sphere_coef(p)], [np.zeros(sh.ncoef(p))], [p], [1.0], prm, info=info,
                      near=False)
        d = operators.DropGeom(inputs.sphere_coef(p), p)
        En = sh.sht_inverse(info["En"][0], p, p)
        En_exact = 5.0 * R / (2.0 * R + 3.0) * 0.7 * ((G @ d.x0) * d.n0).sum(axis=0)
        np.testing.assert_allclose(En, En_exact, atol=1e-12)


def test_stokes_rigid_motion_is_a_solution_for_lambda_one_source():
    """Stokes matvec: with lam = 1 there is no double layer, so A u = 2 u exactly; with
    lam != 1 a constant u satisfies (lam+1) c - (lam-1) D[c] = 2 c on the sphere."""
    p = 5
    for lam in (1.0, 4.0):
        sysm = operators.System([operators.DropGeom(inputs.sphere_coef(p), p, lam)])
        c = np.zeros((3, sh.ncoef(p)))
        c[:, 0] = np.array([1.0, -2.0, 0.5]) * math.sqrt(4 * math.pi)
        np.testing.assert_allclose(sysm.stokes_matvec(c.ravel()), 2.0 * c.ravel(), atol=1e-12)


def test_gmres_matches_direct_solve():
    rng = np.random.default_rng(0)
    A = np.eye(60) * 3 + rng.standard_normal((60, 60)) * 0.2
    b = rng.standard_normal(60)
    x, info = gmres.gmres(lambda v: A @ v, b, tol=1e-12, restart=7)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), atol=1e-10)
    assert info["resid"] <= 1e-12
