"""Parity of the forces, rates and time step (Section 1, Algorithm 1) with the FP64 oracle."""
import math
import os

import numpy as np
import pytest

import inputs
from oracle import physics as P, sh

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL64 = 1e-10
TOL32 = 1e-5


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return max(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300),
               np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1811_10270_gb300 as pkg
    if not os.path.exists(pkg.LIB_PATH):
        from paper_1811_10270_gb300 import build
        build.build()
    pkg.lib()
    return pkg


def T(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def two_drops(p=6, seed=2, gap=0.4):
    cfg = inputs.config2(p=p, seed=seed, gap=gap)
    cfg.drops[1].lam = 0.5
    return cfg


def setup(S, cfg, precision, tol=1e-13):
    ctx = S.Context(precision=precision, R=cfg.R, gmres_tol=tol)
    x = T(np.concatenate([d.xcoef.ravel() for d in cfg.drops]))
    ctx.set_drops([d.p for d in cfg.drops], x, [d.lam for d in cfg.drops])
    g = T(np.concatenate([d.gamma_coef for d in cfg.drops]))
    return ctx, x, g


def test_initial_deformation_rate_of_a_sphere_on_gpu(S):
    """dD/dt = D_T / tau_D for a clean spherical drop (see the oracle pin), through shbim_rates."""
    p, R, Q = 10, 0.1, 1.0
    cfg = inputs.config1(p)
    ctx, x, g = setup(S, cfg, S.FP64)
    u = torch.empty(3 * sh.ncoef(p), device="cuda", dtype=torch.float64)
    gE = torch.empty(sh.ncoef(p), device="cuda", dtype=torch.float64)
    ctx.rates(S.phys(R=R, Q=Q, beta=0.0), g, u, gE)
    uv = sh.sht_inverse(u.cpu().numpy().reshape(3, -1), p, p)
    th, ph = sh.grid_points(p)
    n = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    ur = (uv * n).sum(0)
    A = np.stack([np.ones_like(th), 0.5 * (3 * np.cos(th) ** 2 - 1)]).T
    coef, *_ = np.linalg.lstsq(A, ur, rcond=None)
    DT = 9 * (2 + 3 * R + 2 * R * R - 7 * Q) / (32 * (2 + R) ** 2)
    tau = 35 * 5 / 80.0
    assert abs(0.75 * coef[1] - DT / tau) < 1e-10
    ctx.close()


@pytest.mark.parametrize("precision,tol", [(0, TOL64), (1, TOL32), (2, TOL64)])
def test_rates_match_oracle(S, precision, tol):
    cfg = two_drops()
    ps = [d.p for d in cfg.drops]
    lams = [d.lam for d in cfg.drops]
    prm = P.Params(R=cfg.R, Q=cfg.Q, Ca_E=0.1, beta=0.2, x_s=0.5, E_u=(0.2, 0.0, 1.0), gmres_tol=1e-13)
    u_ref, g_ref = P.rates([d.xcoef for d in cfg.drops], [d.gamma_coef for d in cfg.drops], ps, lams, prm)
    ctx, x, g = setup(S, cfg, precision)
    nc = sum(sh.ncoef(p) for p in ps)
    u = torch.empty(3 * nc, device="cuda", dtype=torch.float64)
    gE = torch.empty(nc, device="cuda", dtype=torch.float64)
    ctx.rates(S.phys(R=cfg.R, Q=cfg.Q, Ca_E=0.1, beta=0.2, x_s=0.5, E_u=(0.2, 0.0, 1.0), inner_tol=1e-6),
              g, u, gE)
    assert rel_err(u.cpu().numpy(), np.concatenate([a.ravel() for a in u_ref])) < tol
    assert rel_err(gE.cpu().numpy(), np.concatenate(g_ref)) < tol
    ctx.close()


def test_field_shape_rates_match_oracle(S):
    """The quadrupole field of Section 3, E_q (-x, -y, 2z) (shbim_set_field_shape with
    diag(-1, -1, 2)), and a random symmetric traceless shape, through shbim_rates against the oracle
    (FP64), plus the unit-sphere closed form E_n = 5R/(2R+3) E_q n.Gn through shbim_electric_rhs."""
    cfg = two_drops()
    ps = [d.p for d in cfg.drops]
    lams = [d.lam for d in cfg.drops]
    rng = np.random.default_rng(11)
    A = rng.standard_normal((3, 3))
    Gr = A + A.T
    Gr -= np.trace(Gr) / 3.0 * np.eye(3)
    for G in (np.diag([-1.0, -1.0, 2.0]), Gr):
        prm = P.Params(R=cfg.R, Q=cfg.Q, Ca_E=0.1, beta=0.2, x_s=0.5, E_u=(0.0, 0.1, 0.0), E_q=0.8,
                       E_G=tuple(map(tuple, G)), gmres_tol=1e-13)
        u_ref, g_ref = P.rates([d.xcoef for d in cfg.drops], [d.gamma_coef for d in cfg.drops], ps, lams, prm)
        ctx, x, g = setup(S, cfg, S.FP64)
        ctx.set_field_shape(G)
        nc = sum(sh.ncoef(p) for p in ps)
        u = torch.empty(3 * nc, device="cuda", dtype=torch.float64)
        gE = torch.empty(nc, device="cuda", dtype=torch.float64)
        ctx.rates(S.phys(R=cfg.R, Q=cfg.Q, Ca_E=0.1, beta=0.2, x_s=0.5, E_u=(0.0, 0.1, 0.0), E_q=0.8), g, u, gE)
        assert rel_err(u.cpu().numpy(), np.concatenate([a.ravel() for a in u_ref])) < TOL64
        assert rel_err(gE.cpu().numpy(), np.concatenate(g_ref)) < TOL64
        ctx.close()
    p, R = 12, 2.0
    ctx = S.Context(precision=S.FP64, R=R, gmres_tol=1e-13)
    ctx.set_drops([p], T(inputs.sphere_coef(p).ravel()), [1.0])
    ctx.set_field_shape(Gr)
    b = torch.empty(sh.ncoef(p), device="cuda", dtype=torch.float64)
    ctx.electric_rhs((0.0, 0.0, 0.0), b, E_q=0.8)
    En = torch.empty_like(b)
    ctx.gmres_solve(S.SYS_ELECTRIC, b, En)
    th, ph = sh.grid_points(p)
    n = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    expect = 0.8 * 5 * R / (2 * R + 3) * (n * (Gr @ n)).sum(axis=0)
    assert np.abs(sh.sht_inverse(En.cpu().numpy(), p, p) - expect).max() < 1e-11
    for bad in (np.diag([1.0, 1.0, 1.0]), np.array([[0, 1.0, 0], [0, 0, 0], [0, 0, 0]])):
        with pytest.raises(S.ShbimError):
            ctx.set_field_shape(bad)
    ctx.close()


@pytest.mark.parametrize("precision", [0, 2])
def test_stokes_rhs_matches_oracle(S, precision):
    """shbim_stokes_rhs for the oracle's E_n: -sum_j S_j[f/Ca_E - f^E] with the charge potential, the
    electric and the Langmuir tractions of Section 1, against the oracle's right-hand side."""
    from oracle import operators
    cfg = two_drops()
    ps = [d.p for d in cfg.drops]
    lams = [d.lam for d in cfg.drops]
    prm = P.Params(R=cfg.R, Q=cfg.Q, Ca_E=0.1, beta=0.2, x_s=0.5, E_u=(0.2, 0.0, 1.0), gmres_tol=1e-13)
    info = {}
    P.rates([d.xcoef for d in cfg.drops], [d.gamma_coef for d in cfg.drops], ps, lams, prm, info=info)
    sysm = operators.System([operators.DropGeom(d.xcoef, d.p, d.lam) for d in cfg.drops], near=True)
    ref = -np.concatenate([a.ravel() for a in sysm.stokes_coef(info["traction"], None)])
    ctx, x, g = setup(S, cfg, precision)
    En = T(np.concatenate(info["En"]))
    out = torch.empty(3 * En.numel(), device="cuda", dtype=torch.float64)
    ctx.stokes_rhs(S.phys(R=cfg.R, Q=cfg.Q, Ca_E=0.1, beta=0.2, x_s=0.5, E_u=(0.2, 0.0, 1.0)), g, En, out)
    assert rel_err(out.cpu().numpy(), ref) < TOL64
    ctx.close()


@pytest.fixture(scope="module")
def rates_p12_gap01():
    """Two drops of degree 12, 0.1 apart (near pairs on both sides), and the oracle's rates."""
    cfg = two_drops(p=12, seed=2, gap=0.1)
    ps = [d.p for d in cfg.drops]
    lams = [d.lam for d in cfg.drops]
    prm = P.Params(R=cfg.R, Q=cfg.Q, Ca_E=0.1, beta=0.2, x_s=0.5, E_u=(0.2, 0.0, 1.0), gmres_tol=1e-13)
    u_ref, g_ref = P.rates([d.xcoef for d in cfg.drops], [d.gamma_coef for d in cfg.drops], ps, lams, prm)
    return cfg, np.concatenate([a.ravel() for a in u_ref]), np.concatenate(g_ref)


@pytest.mark.parametrize("precision,tol", [(1, TOL32), (2, TOL64)])
def test_rates_close_drops_match_oracle(S, rates_p12_gap01, precision, tol):
    """shbim_rates at p = 12 with the drops 0.1 apart (nearly-singular correction active): mixed
    precision (FP32 compensated inner solves refined to an FP64-class residual, one-shot
    applications double-float) and double-float sums, against the FP64 oracle."""
    cfg, u_ref, g_ref = rates_p12_gap01
    ctx, x, g = setup(S, cfg, precision, tol=1e-12)
    assert ctx.near_pairs() > 0
    nc = sum(sh.ncoef(d.p) for d in cfg.drops)
    u = torch.empty(3 * nc, device="cuda", dtype=torch.float64)
    gE = torch.empty(nc, device="cuda", dtype=torch.float64)
    ctx.rates(S.phys(R=cfg.R, Q=cfg.Q, Ca_E=0.1, beta=0.2, x_s=0.5, E_u=(0.2, 0.0, 1.0), inner_tol=1e-5),
              g, u, gE)
    assert rel_err(u.cpu().numpy(), u_ref) < tol
    assert rel_err(gE.cpu().numpy(), g_ref) < tol
    ctx.close()


def test_step_matches_oracle(S):
    cfg = two_drops(p=5, seed=4, gap=0.5)
    ps = [d.p for d in cfg.drops]
    lams = [d.lam for d in cfg.drops]
    prm = P.Params(R=cfg.R, Q=cfg.Q, Ca_E=0.1, beta=0.2, x_s=0.5, E_u=(0.0, 0.0, 1.0), gmres_tol=1e-13)
    dt = 0.02
    xn, gn, err, _ = P.step([d.xcoef for d in cfg.drops], [d.gamma_coef for d in cfg.drops], ps, lams, dt, prm)
    ctx, x, g = setup(S, cfg, S.FP64)
    xo = torch.empty_like(x)
    go = torch.empty_like(g)
    e, its = ctx.step(S.phys(R=cfg.R, Q=cfg.Q, Ca_E=0.1, beta=0.2, x_s=0.5), x, g, dt, xo, go)
    assert rel_err(xo.cpu().numpy(), np.concatenate([a.ravel() for a in xn])) < TOL64
    assert rel_err(go.cpu().numpy(), np.concatenate(gn)) < TOL64
    assert abs(e - err) < 1e-9 * err
    assert min(its) > 0
    ctx.close()


def test_adaptive_steps_conserve_surfactant(S):
    """A few accepted steps with the paper's controller (accept if err < tol,
    dt <- dt (0.9 tol/err)^(1/2)): surfactant mass drifts by far less than the tolerance."""
    cfg = two_drops(p=6, seed=5, gap=0.4)
    ps = [d.p for d in cfg.drops]
    ctx, x, g = setup(S, cfg, S.FP32_COMP, tol=1e-10)
    ph = S.phys(R=cfg.R, Q=cfg.Q, Ca_E=0.1, beta=0.2, x_s=0.5)
    m0 = sum(P.surfactant_mass(d.xcoef, d.gamma_coef, d.p) for d in cfg.drops)
    tol, dt, accepted = 1e-4, 0.01, 0
    for _ in range(12):
        xo, go = torch.empty_like(x), torch.empty_like(g)
        err, _ = ctx.step(ph, x, g, dt, xo, go)
        if err < tol:
            x, g = xo, go
            accepted += 1
        dt = dt * math.sqrt(0.9 * tol / err)
        if accepted >= 4:
            break
    assert accepted >= 4
    xs = x.cpu().numpy()
    gs = g.cpu().numpy()
    off, m1 = 0, 0.0
    for p in ps:
        nc = sh.ncoef(p)
        m1 += P.surfactant_mass(xs[3 * off:3 * off + 3 * nc].reshape(3, nc), gs[off:off + nc], p)
        off += nc
    assert abs(m1 - m0) / m0 < 1e-5
    ctx.close()


def _per_drop(v, ps):
    out, off = [], 0
    for p in ps:
        nc = sh.ncoef(p)
        out.append(v[off:off + nc])
        off += nc
    return out


def test_laplace_beltrami_matches_oracle(S):
    """shbim_laplace_beltrami against the oracle's chart formula on two perturbed drops."""
    cfg = two_drops(p=7, seed=6, gap=0.5)
    ps = [d.p for d in cfg.drops]
    ctx, x, g = setup(S, cfg, S.FP64)
    rng = np.random.default_rng(11)
    f = [rng.standard_normal(sh.ncoef(p)) / (1.0 + np.repeat(np.arange(p + 1), 2 * np.arange(p + 1) + 1))
         for p in ps]
    out = torch.empty(sum(sh.ncoef(p) for p in ps), device="cuda", dtype=torch.float64)
    ctx.laplace_beltrami(T(np.concatenate(f)), out)
    ref = [P.SurfaceGrid(d.xcoef, d.p, 2 * d.p + 1).project(
        P.SurfaceGrid(d.xcoef, d.p, 2 * d.p + 1).laplace_beltrami(fi)) for d, fi in zip(cfg.drops, f)]
    assert rel_err(out.cpu().numpy(), np.concatenate(ref)) < TOL64
    ctx.close()


@pytest.mark.parametrize("with_x0", [False, True])
def test_diffusion_solve_matches_oracle(S, with_x0):
    """(I - c Delta_S) G = b by the right-preconditioned GMRES of SHBIM_SYS_DIFFUSION."""
    cfg = two_drops(p=6, seed=7, gap=0.5)
    ps = [d.p for d in cfg.drops]
    ctx, x, g = setup(S, cfg, S.FP64)
    c = 0.05
    ctx.set_diffusion(c)
    rhs = np.concatenate([d.gamma_coef for d in cfg.drops])
    ref = np.concatenate([P.diffusion_solve(d.xcoef, d.p, d.gamma_coef, c) for d in cfg.drops])
    out = torch.empty(len(rhs), device="cuda", dtype=torch.float64)
    x0 = T(rhs) if with_x0 else None
    its, res = ctx.gmres_solve(S.SYS_DIFFUSION, T(rhs), out, x0=x0)
    assert res < 1e-12
    assert rel_err(out.cpu().numpy(), ref) < TOL64
    # the preconditioner is the exact inverse on a sphere: few iterations on these shapes
    assert its < 20
    ctx.close()


@pytest.mark.parametrize("precision,tol", [(0, TOL64), (1, TOL32)])
def test_step_with_diffusion_matches_oracle(S, precision, tol):
    """IMEX step of Algorithm 1 at a finite Peclet number."""
    cfg = two_drops(p=5, seed=8, gap=0.5)
    ps = [d.p for d in cfg.drops]
    lams = [d.lam for d in cfg.drops]
    Pe = 10.0
    prm = P.Params(R=cfg.R, Q=cfg.Q, Ca_E=0.1, beta=0.2, x_s=0.5, gmres_tol=1e-13, Pe=Pe)
    dt = 0.02
    xn, gn, err, _ = P.step([d.xcoef for d in cfg.drops], [d.gamma_coef for d in cfg.drops], ps, lams, dt, prm)
    ctx, x, g = setup(S, cfg, precision)
    xo = torch.empty_like(x)
    go = torch.empty_like(g)
    e, its = ctx.step(S.phys(R=cfg.R, Q=cfg.Q, Ca_E=0.1, beta=0.2, x_s=0.5, inner_tol=1e-6, Pe=Pe),
                      x, g, dt, xo, go)
    assert rel_err(xo.cpu().numpy(), np.concatenate([a.ravel() for a in xn])) < tol
    assert rel_err(go.cpu().numpy(), np.concatenate(gn)) < tol
    assert abs(e - err) < max(1e-9, tol) * err
    # diffusion changes the surfactant increment by far more than the tolerance
    xi, gi, _, _ = P.step([d.xcoef for d in cfg.drops], [d.gamma_coef for d in cfg.drops], ps, lams, dt,
                          P.Params(R=cfg.R, Q=cfg.Q, Ca_E=0.1, beta=0.2, x_s=0.5, gmres_tol=1e-13))
    g0 = np.concatenate([d.gamma_coef for d in cfg.drops])
    assert rel_err(np.concatenate(gi) - g0, np.concatenate(gn) - g0) > 0.01
    assert rel_err(go.cpu().numpy() - g0, np.concatenate(gn) - g0) < 1e3 * tol
    ctx.close()


def test_negative_peclet_is_rejected(S):
    cfg = two_drops(p=4, seed=9, gap=0.5)
    ctx, x, g = setup(S, cfg, S.FP64)
    xo, go = torch.empty_like(x), torch.empty_like(g)
    with pytest.raises(S.ShbimError):
        ctx.step(S.phys(R=cfg.R, Pe=-1.0), x, g, 0.01, xo, go)
    with pytest.raises(S.ShbimError):
        ctx.set_diffusion(-0.5)
    ctx.close()
