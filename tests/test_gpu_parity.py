"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded inputs.

Tolerances (relative L2 and relative max, each quantity): 1e-10 for the FP64 path, 1e-5 for
the FP32 compensated all-pairs path.
"""
import math
import os

import numpy as np
import pytest

import inputs
from oracle import geometry, gmres, operators, sh

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL64 = 1e-10
TOL32 = 1e-5


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    l2 = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
    mx = np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)
    return max(l2, mx)


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


DEV = "cuda"


def T(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def make(S, drops, precision, R=2.0, near=True):
    ctx = S.Context(precision=precision, R=R, gmres_tol=1e-12)
    ctx.set_near(near)
    xc = T(np.concatenate([d.xcoef.ravel() for d in drops]))
    ctx.set_drops([d.p for d in drops], xc, [d.lam for d in drops])
    return ctx


def oracle_system(drops, near=True):
    """Oracle operators; near=True applies the same nearly-singular correction as the library."""
    return operators.System([operators.DropGeom(d.xcoef, d.p, d.lam) for d in drops], near=near)


def split_grid(vec, drops, ncomp):
    out, o = [], 0
    for d in drops:
        k = ncomp * sh.npts(d.p) if hasattr(sh, "npts") else ncomp * (d.p + 1) * (2 * d.p + 2)
        out.append(vec[o:o + k].reshape(ncomp, -1) if ncomp > 1 else vec[o:o + k])
        o += k
    return out


# --------------------------------------------------------------------------- transforms

@pytest.mark.parametrize("p", [1, 5, 16])
def test_sht_matches_oracle(S, p):
    d = inputs.config1(p).drops[0]
    ctx = make(S, [d], S.FP64)
    rng = np.random.default_rng(p)
    c = rng.standard_normal((3, sh.ncoef(p)))
    for grid, q in ((S.GRID_BASE, p), (S.GRID_UP, 2 * p + 1)):
        n = (q + 1) * (2 * q + 2)
        out = torch.empty(3 * n, device=DEV, dtype=torch.float64)
        ctx.sht(S.SHT_INVERSE, grid, [0, 0, 0], T(c), out)
        assert rel_err(out.cpu().numpy().reshape(3, n), sh.sht_inverse(c, p, q)) < 1e-12
        g = rng.standard_normal((3, n))
        cf = torch.empty(3 * sh.ncoef(p), device=DEV, dtype=torch.float64)
        ctx.sht(S.SHT_FORWARD, grid, [0, 0, 0], T(g), cf)
        assert rel_err(cf.cpu().numpy().reshape(3, -1), sh.sht_forward(g, p, q)) < 1e-12
    ctx.close()


def test_sht_field_drop_map_matches_oracle(S):
    """Fields of drops of different degrees in one call, in the order the drop map gives
    (drop 1, drop 0, drop 1): each field is transformed on its own drop's grid."""
    cfg = inputs.config2(p=4, seed=2, gap=0.3)
    d0 = cfg.drops[0]
    d1 = inputs.Drop(7, inputs.perturbed_coef(7, np.random.default_rng(3), 1.0, (0.0, 0.0, 3.0)),
                     np.zeros(sh.ncoef(7)), 1.0, np.zeros(3), 1.0)
    ctx = make(S, [d0, d1], S.FP64)
    fd = [1, 0, 1]
    ps = [[4, 7][i] for i in fd]
    rng = np.random.default_rng(9)
    for grid in (S.GRID_BASE, S.GRID_UP):
        qs = [p if grid == S.GRID_BASE else 2 * p + 1 for p in ps]
        cs = [rng.standard_normal(sh.ncoef(p)) for p in ps]
        out = torch.empty(sum((q + 1) * (2 * q + 2) for q in qs), device=DEV, dtype=torch.float64)
        ctx.sht(S.SHT_INVERSE, grid, fd, T(np.concatenate(cs)), out)
        ref = np.concatenate([sh.sht_inverse(c[None], p, q)[0] for c, p, q in zip(cs, ps, qs)])
        assert rel_err(out.cpu().numpy(), ref) < 1e-12
        gs = [rng.standard_normal((q + 1) * (2 * q + 2)) for q in qs]
        cf = torch.empty(sum(sh.ncoef(p) for p in ps), device=DEV, dtype=torch.float64)
        ctx.sht(S.SHT_FORWARD, grid, fd, T(np.concatenate(gs)), cf)
        ref = np.concatenate([sh.sht_forward(g[None], p, q)[0] for g, p, q in zip(gs, ps, qs)])
        assert rel_err(cf.cpu().numpy(), ref) < 1e-12
    ctx.close()


def test_target_geometry_matches_oracle(S):
    p = 9
    xc = inputs.perturbed_coef(p, np.random.default_rng(11), 1.1, (0.3, -0.2, 0.5))
    d = inputs.Drop(p, xc, np.zeros(sh.ncoef(p)), 1.0, np.zeros(3), 1.0)
    ctx = make(S, [d], S.FP64)
    nt = (p + 1) * (2 * p + 2)
    g = torch.empty(7 * nt, device=DEV, dtype=torch.float64)
    ctx.target_geometry(g)
    g = g.cpu().numpy().reshape(7, nt)
    x, n, J = geometry.surface_on_grid(xc, p, p)
    assert rel_err(g[0:3], x) < 1e-12
    assert rel_err(g[3:6], n) < 1e-12
    assert rel_err(g[6], J) < 1e-12
    ctx.close()


# --------------------------------------------------------------------------- closed forms

@pytest.mark.parametrize("p", [1, 16, 64])
def test_single_layer_eigenrelation_unit_sphere(S, p):
    """(1/4pi) int Y_lm / r = Y_lm/(2l+1) on the unit sphere; the target-normal double layer
    is half of it there. p = 64 is the largest degree the library accepts."""
    d = inputs.config1(p).drops[0]
    ctx = make(S, [d], S.FP64)
    rng = np.random.default_rng(3)
    sig = inputs.random_density(p, rng)[0]
    scale = np.array([1.0 / (2 * n + 1) for n in range(p + 1) for _ in range(2 * n + 1)])
    nt = (p + 1) * (2 * p + 2)
    out = torch.empty(nt, device=DEV, dtype=torch.float64)
    ctx.eval_electric(S.LAPLACE_SL, T(sig), out, S.OUT_GRID)
    expect = sh.sht_inverse(sig * scale, p, p) if p <= 32 else None
    got = out.cpu().numpy()
    coef = torch.empty(sh.ncoef(p), device=DEV, dtype=torch.float64)
    ctx.eval_electric(S.LAPLACE_SL, T(sig), coef, S.OUT_COEF)
    assert rel_err(coef.cpu().numpy(), sig * scale) < TOL64
    if expect is not None:
        assert rel_err(got, expect) < TOL64
    ctx.eval_electric(S.LAPLACE_DL, T(sig), coef, S.OUT_COEF)
    assert rel_err(coef.cpu().numpy(), 0.5 * sig * scale) < TOL64
    ctx.close()


def test_stokes_identities_unit_sphere(S):
    """S[c] = (4/3) c, D[c] = c (as (lam-1) D with lam = 2) and S[n] = 0 on the unit sphere."""
    p = 12
    d = inputs.config1(p).drops[0]
    d.lam = 2.0
    ctx = make(S, [d], S.FP64)
    nc = sh.ncoef(p)
    c = np.zeros((3, nc))
    c[:, 0] = np.array([0.3, -0.7, 1.1]) * math.sqrt(4 * math.pi)
    out = torch.empty(3 * nc, device=DEV, dtype=torch.float64)
    ctx.eval_stokes(T(c), None, out)
    assert rel_err(out.cpu().numpy(), 4.0 / 3.0 * c.ravel()) < TOL64
    ctx.eval_stokes(None, T(c), out)
    assert rel_err(out.cpu().numpy(), c.ravel()) < TOL64
    ctx.eval_stokes(T(inputs.sphere_coef(p)), None, out)
    assert np.abs(out.cpu().numpy()).max() < 1e-12
    ctx.close()


# --------------------------------------------------------------------------- full parity

def _two_drop_cfg(p, seed=0, gap=0.3):
    cfg = inputs.config2(p=p, seed=seed, gap=gap)
    cfg.drops[1].lam = 0.5
    return cfg


@pytest.fixture(scope="module")
def two_drops_p12():
    """Two perturbed drops at p = 12: 338 targets per drop = two pair tiles with a ragged tail."""
    cfg = _two_drop_cfg(12)
    return cfg, oracle_system(cfg.drops)


@pytest.mark.parametrize("precision,tol", [(0, TOL64), (1, TOL32), (2, TOL64)])
def test_laplace_two_drops_matches_oracle(S, two_drops_p12, precision, tol):
    cfg, sysm = two_drops_p12
    ctx = make(S, cfg.drops, precision, cfg.R)
    rng = np.random.default_rng(5)
    sig = [inputs.random_density(d.p, rng)[0] for d in cfg.drops]
    nc_tot = sum(sh.ncoef(d.p) for d in cfg.drops)
    nt_tot = sum((d.p + 1) * (2 * d.p + 2) for d in cfg.drops)
    for which, kind in ((S.LAPLACE_DL, "ladl"), (S.LAPLACE_SL, "lsl")):
        out = torch.empty(nt_tot, device=DEV, dtype=torch.float64)
        ctx.eval_electric(which, T(np.concatenate(sig)), out, S.OUT_GRID)
        assert rel_err(out.cpu().numpy(), np.concatenate(sysm.laplace_grid(kind, sig))) < tol
        co = torch.empty(nc_tot, device=DEV, dtype=torch.float64)
        ctx.eval_electric(which, T(np.concatenate(sig)), co, S.OUT_COEF)
        assert rel_err(co.cpu().numpy(), np.concatenate(sysm.laplace_coef(kind, sig))) < tol
    ctx.close()


@pytest.mark.parametrize("precision,tol", [(0, TOL64), (1, TOL32), (2, TOL64)])
def test_stokes_two_drops_matches_oracle(S, two_drops_p12, precision, tol):
    cfg, sysm = two_drops_p12
    ctx = make(S, cfg.drops, precision, cfg.R)
    rng = np.random.default_rng(6)
    f = [inputs.random_density(d.p, rng, 3) for d in cfg.drops]
    u = [inputs.random_density(d.p, rng, 3) for d in cfg.drops]
    F = T(np.concatenate([a.ravel() for a in f]))
    U = T(np.concatenate([a.ravel() for a in u]))
    nt_tot = sum((d.p + 1) * (2 * d.p + 2) for d in cfg.drops)
    nc_tot = sum(sh.ncoef(d.p) for d in cfg.drops)
    for ff, uu, fo, uo in ((F, U, f, u), (F, None, f, None), (None, U, None, u)):
        out = torch.empty(3 * nt_tot, device=DEV, dtype=torch.float64)
        ctx.eval_stokes(ff, uu, out, S.OUT_GRID)
        ref = np.concatenate([a.ravel() for a in sysm.stokes_grid(fo, uo)])
        assert rel_err(out.cpu().numpy(), ref) < tol
        co = torch.empty(3 * nc_tot, device=DEV, dtype=torch.float64)
        ctx.eval_stokes(ff, uu, co, S.OUT_COEF)
        ref = np.concatenate([a.ravel() for a in sysm.stokes_coef(fo, uo)])
        assert rel_err(co.cpu().numpy(), ref) < tol
    ctx.close()


def test_three_drops_uneven_degrees_match_oracle(S):
    rng = np.random.default_rng(9)
    drops = []
    for p, ctr, lam in ((4, (0, 0, 0), 3.0), (7, (2.6, 0.1, 0.2), 1.0), (5, (-0.3, 2.5, -0.4), 0.7)):
        drops.append(inputs.Drop(p, inputs.perturbed_coef(p, rng, 1.0, ctr), np.zeros(sh.ncoef(p)),
                                 lam, np.asarray(ctr, float), 1.0))
    sysm = oracle_system(drops)
    sig = [inputs.random_density(d.p, rng)[0] for d in drops]
    u = [inputs.random_density(d.p, rng, 3) for d in drops]
    nc_tot = sum(sh.ncoef(d.p) for d in drops)
    for precision, tol in ((S.FP64, TOL64), (S.FP32_COMP, TOL32), (S.DF64, TOL64)):
        ctx = make(S, drops, precision)
        co = torch.empty(nc_tot, device=DEV, dtype=torch.float64)
        ctx.eval_electric(S.LAPLACE_DL, T(np.concatenate(sig)), co, S.OUT_COEF)
        assert rel_err(co.cpu().numpy(), np.concatenate(sysm.laplace_coef("ladl", sig))) < tol
        co3 = torch.empty(3 * nc_tot, device=DEV, dtype=torch.float64)
        ctx.eval_stokes(T(np.concatenate([a.ravel() for a in u])), T(np.concatenate([a.ravel() for a in u])),
                        co3, S.OUT_COEF)
        ref = np.concatenate([a.ravel() for a in sysm.stokes_coef(u, u)])
        assert rel_err(co3.cpu().numpy(), ref) < tol
        ctx.close()


def test_double_float_singular_rows_match_fp64_rows_and_oracle(S):
    """The singular self rows built in double-float arithmetic (the default, with the Fourier and
    Legendre stages and the rotations on the tensor cores; subsets; none) against the rows of the
    FP64 build and the oracle, on one perturbed drop (self term only) and on two drops."""
    rng = np.random.default_rng(31)
    one = [inputs.Drop(11, inputs.perturbed_coef(11, rng, 1.0, (0.1, -0.2, 0.3)), np.zeros(sh.ncoef(11)),
                       2.5, np.array([0.1, -0.2, 0.3]), 1.0)]
    two = _two_drop_cfg(8, seed=3, gap=0.3).drops
    for drops in (one, two):
        sysm = oracle_system(drops)
        nc = sum(sh.ncoef(d.p) for d in drops)
        sig = [inputs.random_density(d.p, rng)[0] for d in drops]
        u = [inputs.random_density(d.p, rng, 3) for d in drops]
        res = {}
        variants = ((S.FP64, 0), (S.DF64, 0), (S.DF64, S.TC_FOURIER), (S.DF64, S.TC_FOURIER | S.TC_LEGENDRE),
                    (S.DF64, S.TC_ROTATION), (S.DF64, S.TC_ALL))
        for rows, tc in variants:
            ctx = S.Context(precision=S.FP64, R=2.0, gmres_tol=1e-12)
            ctx.set_rows_precision(rows)
            ctx.set_tensor_cores(tc)
            ctx.set_drops([d.p for d in drops], T(np.concatenate([d.xcoef.ravel() for d in drops])),
                          [d.lam for d in drops])
            out = []
            for which in (S.LAPLACE_DL, S.LAPLACE_SL):
                o = torch.empty(nc, device=DEV, dtype=torch.float64)
                ctx.eval_electric(which, T(np.concatenate(sig)), o, S.OUT_COEF)
                out.append(o.cpu().numpy())
            o3 = torch.empty(3 * nc, device=DEV, dtype=torch.float64)
            U = T(np.concatenate([a.ravel() for a in u]))
            ctx.eval_stokes(U, U, o3, S.OUT_COEF)
            out.append(o3.cpu().numpy())
            res[(rows, tc)] = out
            ctx.close()
        refs = [np.concatenate(sysm.laplace_coef("ladl", sig)), np.concatenate(sysm.laplace_coef("lsl", sig)),
                np.concatenate([a.ravel() for a in sysm.stokes_coef(u, u)])]
        for key in variants[1:]:
            for a, b, ref in zip(res[key], res[(S.FP64, 0)], refs):
                assert rel_err(a, b) < 1e-11, key
                assert rel_err(a, ref) < TOL64, key


def test_quantized_double_float_pairs_match_fp64(S):
    """The FP64-class pair sums on quantised positions (shbim_set_quantized_pairs, the default) and the
    general double-float form against native FP64 sums, target by target on the grid, for every kernel
    kind (Laplace DL and SL, Stokes S + D, S alone, D alone): two drops 0.1 apart (close pairs, ragged
    tiles) and six small drops spread over a 40-wide box (a coarse quantum: the largest offsets set it).
    Both forms stay within the FP64 tolerance (about 1e-11 of the largest value is measured with these
    oscillating densities, whose terms cancel), and the quantised form is not much less accurate than
    the general one."""
    rng = np.random.default_rng(41)
    close = _two_drop_cfg(12, seed=5, gap=0.1).drops
    spread = []
    for k, ctr in enumerate(((0, 0, 0), (19.0, -3.0, 1.0), (-18.5, 4.0, 2.0), (2.0, 19.5, -1.0),
                             (1.0, -19.0, 18.0), (3.1, 0.2, -0.4))):
        p = 4 + k
        spread.append(inputs.Drop(p, inputs.perturbed_coef(p, rng, 1.0, ctr), np.zeros(sh.ncoef(p)),
                                  0.5 + k, np.asarray(ctr, float), 1.0))
    for drops in (close, spread):
        nt = sum((d.p + 1) * (2 * d.p + 2) for d in drops)
        sig = T(np.concatenate([inputs.random_density(d.p, rng)[0] for d in drops]))
        F = T(np.concatenate([inputs.random_density(d.p, rng, 3).ravel() for d in drops]))
        U = T(np.concatenate([inputs.random_density(d.p, rng, 3).ravel() for d in drops]))
        res = {}
        for key, prec, dq in (("fp64", S.FP64, True), ("df", S.DF64, False), ("dq", S.DF64, True)):
            ctx = make(S, drops, prec, near=False)
            ctx.set_quantized_pairs(dq)
            outs = []
            for which in (S.LAPLACE_DL, S.LAPLACE_SL):
                o = torch.empty(nt, device=DEV, dtype=torch.float64)
                ctx.eval_electric(which, sig, o, S.OUT_GRID)
                outs.append(o.cpu().numpy())
            for f, u in ((F, U), (F, None), (None, U)):
                o = torch.empty(3 * nt, device=DEV, dtype=torch.float64)
                ctx.eval_stokes(f, u, o, S.OUT_GRID)
                outs.append(o.cpu().numpy())
            res[key] = outs
            ctx.close()
        for k, (a, b, c) in enumerate(zip(res["dq"], res["fp64"], res["df"])):
            e_dq, e_df = rel_err(a, b), rel_err(c, b)
            assert e_dq < TOL64 and e_df < TOL64, (k, e_dq, e_df)
            assert e_dq < 10.0 * e_df + 1e-12, (k, e_dq, e_df)


def test_every_pair_launch_shape_matches_oracle(S):
    """Each register blocking (1, 2, 4 targets per thread) with one and several source splits, as
    a CTA per work unit and as persistent CTAs on the work counter (the same sums to the bit, also
    on a second launch after the counter reset): drops of 200, 98 and 50 targets leave ragged and
    empty sub-tiles in every shape."""
    rng = np.random.default_rng(21)
    drops = []
    for p, ctr, lam in ((9, (0, 0, 0), 2.0), (6, (2.4, 0.3, -0.2), 0.5), (4, (-0.4, -2.3, 0.5), 4.0)):
        drops.append(inputs.Drop(p, inputs.perturbed_coef(p, rng, 1.0, ctr), np.zeros(sh.ncoef(p)),
                                 lam, np.asarray(ctr, float), 1.0))
    sysm = oracle_system(drops, near=False)
    sig = [inputs.random_density(d.p, rng)[0] for d in drops]
    u = [inputs.random_density(d.p, rng, 3) for d in drops]
    f = [inputs.random_density(d.p, rng, 3) for d in drops]
    ref = {0: np.concatenate(sysm.laplace_coef("ladl", sig)), 1: np.concatenate(sysm.laplace_coef("lsl", sig)),
           2: np.concatenate([a.ravel() for a in sysm.stokes_coef(f, u)]),
           3: np.concatenate([a.ravel() for a in sysm.stokes_coef(f, None)]),
           4: np.concatenate([a.ravel() for a in sysm.stokes_coef(None, u)])}
    nc = sum(sh.ncoef(d.p) for d in drops)
    ctx = make(S, drops, S.FP32_COMP, near=False)
    sig_d = T(np.concatenate(sig))
    f_d = T(np.concatenate([a.ravel() for a in f]))
    u_d = T(np.concatenate([a.ravel() for a in u]))
    _, default_splits, fixed = ctx.pair_shape(2)
    assert not fixed                      # nothing launched yet: the shape is not chosen
    for tpt in (1, 2, 4):
        for splits in sorted({1, max(1, default_splits)}):
            got = {}
            for queue in (False, True):
                for kind in (0, 1, 2, 3, 4):
                    ctx.set_pair_shape(kind, tpt, splits)
                    ctx.set_pair_queue(kind, queue)
                    assert ctx.pair_shape(kind) == (tpt, splits, True) and ctx.pair_queue(kind) == queue
                outs = []
                for rep in range(2 if queue else 1):
                    out = torch.empty(nc, device=DEV, dtype=torch.float64)
                    ctx.eval_electric(S.LAPLACE_DL, sig_d, out, S.OUT_COEF)
                    dl = out.cpu().numpy()
                    ctx.eval_electric(S.LAPLACE_SL, sig_d, out, S.OUT_COEF)
                    sl = out.cpu().numpy()
                    out3 = torch.empty(3 * nc, device=DEV, dtype=torch.float64)
                    ctx.eval_stokes(f_d, u_d, out3, S.OUT_COEF)
                    sd = out3.cpu().numpy()
                    ctx.eval_stokes(f_d, None, out3, S.OUT_COEF)
                    so = out3.cpu().numpy()
                    ctx.eval_stokes(None, u_d, out3, S.OUT_COEF)
                    outs.append((dl, sl, sd, so, out3.cpu().numpy()))
                    for k in range(5):
                        assert rel_err(outs[-1][k], ref[k]) < TOL32, (tpt, splits, queue, k)
                got[queue] = outs
            for a, b in zip(got[False][0], got[True][0]):
                assert np.array_equal(a, b), (tpt, splits)
            for a, b in zip(got[True][0], got[True][1]):
                assert np.array_equal(a, b), (tpt, splits)
    with pytest.raises(S.ShbimError):
        ctx.set_pair_shape(0, 3, 1)
    with pytest.raises(S.ShbimError):
        ctx.set_pair_shape(0, 1, 0)
    ctx.close()
    # the autotuner settles on one of the shapes and keeps the results within tolerance
    ctx = make(S, drops, S.FP32_COMP, near=False)
    out3 = torch.empty(3 * nc, device=DEV, dtype=torch.float64)
    ctx.eval_stokes(f_d, u_d, out3, S.OUT_COEF)
    tpt, splits, fixed = ctx.pair_shape(2)
    assert fixed and tpt in (1, 2, 4) and splits >= 1 and ctx.pair_queue(2) in (False, True)
    assert rel_err(out3.cpu().numpy(), ref[2]) < TOL32
    ctx.close()


@pytest.fixture(scope="module")
def full_size_two_drops():
    """The two-drop workload (p = 32, 0.1 apart) with its oracle and the sampled targets: per drop
    the first and last target, the edges of the 512-target pair tiles and of the 256-target
    launches, the target closest to the gap, and 16 targets spread over the oracle's near list
    (where the upsampled rule replaces the degree-q one)."""
    cfg = inputs.config2(p=32, seed=0, gap=0.1)
    sysm = oracle_system(cfg.drops, near=True)
    pairs = sysm.near_pairs()
    nt = (32 + 1) * 66
    picks = [0, 255, 256, 511, 512, 1023, 1024, 2047, 2048, nt - 1]
    sel = []
    for i, dg in enumerate(sysm.drops):
        near_t = sorted({t for (ii, t, j) in pairs if ii == i})
        assert len(near_t) >= 16
        spread = [near_t[k] for k in np.linspace(0, len(near_t) - 1, 16).astype(int)]
        gap_t = int(np.argmin(np.abs(dg.x0[2])))
        sel.append(sorted(set(picks + spread + [gap_t])))
    rng = np.random.default_rng(12)
    sig = [inputs.random_density(d.p, rng)[0] for d in cfg.drops]
    f = [inputs.random_density(d.p, rng, 3) for d in cfg.drops]
    from oracle import nearsing
    fine = {}
    ref = {}
    for i in range(2):
        ref[("ladl", i)] = nearsing.corrected_laplace_targets(sysm, "ladl", sig, i, sel[i], pairs, fine)
        ref[("lsl", i)] = nearsing.corrected_laplace_targets(sysm, "lsl", sig, i, sel[i], pairs, fine)
        ref[("sto", i)] = nearsing.corrected_stokes_targets(sysm, f, f, i, sel[i], pairs, fine)
    return cfg, sysm, sel, sig, f, ref, len(pairs)


@pytest.mark.parametrize("precision,tol", [(0, TOL64), (1, TOL32), (2, TOL64)])
def test_full_size_two_drops_sampled_targets(S, full_size_two_drops, precision, tol):
    """Two p = 32 drops 0.1 apart (the two-drop workload) in the bench's launch configuration, with
    the nearly-singular correction on (its default): target values of the Laplace double and single
    layers and of the Stokes S[f] + (lambda - 1) D[f] at the sampled targets against the oracle
    evaluated one target at a time, near targets through the oracle's upsampled rule."""
    cfg, sysm, sel, sig, f, ref, npairs = full_size_two_drops
    nt = (32 + 1) * 66
    ctx = make(S, cfg.drops, precision, cfg.R, near=True)
    assert ctx.near_pairs() == npairs
    F = T(np.concatenate([a.ravel() for a in f]))
    for which, kind in ((S.LAPLACE_DL, "ladl"), (S.LAPLACE_SL, "lsl")):
        out = torch.empty(2 * nt, device=DEV, dtype=torch.float64)
        ctx.eval_electric(which, T(np.concatenate(sig)), out, S.OUT_GRID)
        got = out.cpu().numpy()
        for i in range(2):
            assert rel_err(got[i * nt:(i + 1) * nt][sel[i]], ref[(kind, i)]) < tol, (kind, i)
    out3 = torch.empty(6 * nt, device=DEV, dtype=torch.float64)
    ctx.eval_stokes(F, F, out3, S.OUT_GRID)
    got = out3.cpu().numpy()
    for i in range(2):
        assert rel_err(got[3 * i * nt:3 * (i + 1) * nt].reshape(3, nt)[:, sel[i]], ref[("sto", i)]) < tol, i
    ctx.close()


@pytest.fixture(scope="module")
def batched_sampled():
    """The batched workload (64 drops, p 16-48, seed 3) with its oracle and sampled targets: on the first
    drop of each degree, the first and last target and the edges of the 256- and 512-target launches,
    plus up to four targets spread over the drop's near list (where the upsampled rule replaces the
    degree-q one); oracle values of the Laplace double and single layers and of the Stokes
    S[f] + (lambda - 1) D[f] there, one target at a time."""
    from oracle import nearsing
    cfg = inputs.config3(seed=3)
    sysm = oracle_system(cfg.drops, near=True)
    first = {}
    for i, d in enumerate(cfg.drops):
        first.setdefault(d.p, i)
    sel, pairs = {}, []
    for p, i in sorted(first.items()):
        nt = sysm.drops[i].nt
        prs = nearsing.near_pairs_of(sysm, i)
        near_t = sorted({t for (_, t, _) in prs})
        spread = [near_t[k] for k in np.linspace(0, len(near_t) - 1, min(4, len(near_t))).astype(int)] if near_t else []
        sel[i] = sorted(set([0, 255, 256, 511, 512, nt - 1] + spread))
        pairs += [pr for pr in prs if pr[1] in sel[i]]
    assert len(pairs) >= 4
    rng = np.random.default_rng(12)
    sig = [inputs.random_density(d.p, rng)[0] for d in cfg.drops]
    f = [inputs.random_density(d.p, rng, 3) for d in cfg.drops]
    fine, ref = {}, {}
    for i in sel:
        ref[("ladl", i)] = nearsing.corrected_laplace_targets(sysm, "ladl", sig, i, sel[i], pairs, fine)
        ref[("lsl", i)] = nearsing.corrected_laplace_targets(sysm, "lsl", sig, i, sel[i], pairs, fine)
        ref[("sto", i)] = nearsing.corrected_stokes_targets(sysm, f, f, i, sel[i], pairs, fine)
    return cfg, sel, sig, f, ref


# FP64-class bound of the Stokes values at the batched workload: the singular rows (built in double-float
# with tensor-core digit products, ~2^-40 of the sum of magnitudes per entry) give the self stresslet term
# of its first p = 32 drop (lambda = 5.96, self term 80 % of the value) ~1.7e-10 relative with these
# oscillating densities; measured 1.34e-10 for the whole value in FP64 mode
TOL64_BATCHED_STOKES = 5e-10


@pytest.mark.parametrize("precision,tol", [(0, TOL64), (1, TOL32), (2, TOL64)])
def test_batched_workload_sampled_targets(S, batched_sampled, precision, tol):
    """The bench's own workload (64 drops of degree 16-48, near correction on, the launch shapes the
    bench uses) in each precision: target values of the Laplace double and single layers and of the
    Stokes S[f] + (lambda - 1) D[f] at the sampled targets against the oracle (FP64 and FP64-class
    Stokes values within TOL64_BATCHED_STOKES)."""
    cfg, sel, sig, f, ref = batched_sampled
    ctx = make(S, cfg.drops, precision, cfg.R, near=True)
    nc, nt, ns = ctx.sizes()
    offs = np.cumsum([0] + [(d.p + 1) * (2 * d.p + 2) for d in cfg.drops])
    F = T(np.concatenate([a.ravel() for a in f]))
    for which, kind in ((S.LAPLACE_DL, "ladl"), (S.LAPLACE_SL, "lsl")):
        out = torch.empty(nt, device=DEV, dtype=torch.float64)
        ctx.eval_electric(which, T(np.concatenate(sig)), out, S.OUT_GRID)
        got = out.cpu().numpy()
        for i in sel:
            assert rel_err(got[offs[i]:offs[i + 1]][sel[i]], ref[(kind, i)]) < tol, (kind, i)
    out3 = torch.empty(3 * nt, device=DEV, dtype=torch.float64)
    ctx.eval_stokes(F, F, out3, S.OUT_GRID)
    got = out3.cpu().numpy()
    tol_sto = tol if precision == S.FP32_COMP else TOL64_BATCHED_STOKES
    for i in sel:
        n_i = offs[i + 1] - offs[i]
        assert rel_err(got[3 * offs[i]:3 * offs[i + 1]].reshape(3, n_i)[:, sel[i]], ref[("sto", i)]) < tol_sto, i
    ctx.close()


@pytest.mark.parametrize("p", [44, 64])
def test_large_degree_perturbed_drop_matches_oracle(S, p):
    """A perturbed drop above the tensor-core kernels' degree limit (p > 39: the double-float row
    build with the degree-block rotations on the FP32 pipe): Laplace double and single layer and the
    Stokes S[f] + (lambda - 1) D[f] self terms at sampled targets (pole rows, equator, last) against
    the oracle's direct rotated evaluation."""
    from oracle import quadrature
    rng = np.random.default_rng(100 + p)
    ctr = np.array([0.2, -0.1, 0.3])
    d = inputs.Drop(p, inputs.perturbed_coef(p, rng, 1.0, ctr), np.zeros(sh.ncoef(p)), 2.5, ctr, 1.0)
    nt = (p + 1) * (2 * p + 2)
    sel = [0, (p // 2) * (2 * p + 2) + 7, nt // 2 + p, nt - 1]
    sig = inputs.random_density(p, rng)[0]
    f = inputs.random_density(p, rng, 3)
    ctx = make(S, [d], S.FP64, 2.0)
    out = {}
    for which, kind in ((S.LAPLACE_DL, "ladl"), (S.LAPLACE_SL, "lsl")):
        o = torch.empty(nt, device=DEV, dtype=torch.float64)
        ctx.eval_electric(which, T(sig), o, S.OUT_GRID)
        out[kind] = o.cpu().numpy()[sel]
    o3 = torch.empty(3 * nt, device=DEV, dtype=torch.float64)
    ctx.eval_stokes(T(f), T(f), o3, S.OUT_GRID)
    out["sto"] = o3.cpu().numpy().reshape(3, nt)[:, sel]
    ctx.close()
    th, ph = sh.grid_points(p)
    ref = {"ladl": [], "lsl": [], "sto": []}
    for t in sel:
        r = quadrature.self_rows(d.xcoef, p, 2 * p + 1, th[t], ph[t], ["ladl", "lsl", "sto_s", "sto_d"])
        ref["ladl"].append(r["ladl"] @ sig)
        ref["lsl"].append(r["lsl"] @ sig)
        ref["sto"].append(np.einsum("ikc,kc->i", r["sto_s"], f) + (d.lam - 1.0) * np.einsum("ikc,kc->i", r["sto_d"], f))
        del r
    for kind in ("ladl", "lsl"):
        assert rel_err(out[kind], np.array(ref[kind])) < TOL64, kind
    assert rel_err(out["sto"], np.array(ref["sto"]).T) < TOL64


# --------------------------------------------------------------------------- GMRES

def test_gmres_electric_unit_sphere_closed_form(S):
    """Eq. E_n on the unit sphere in a uniform field: E_n = 3R/(R+2) E.n (config: p = 16,
    R = 0.1, E = z)."""
    cfg = inputs.config1(16)
    ctx = make(S, cfg.drops, S.FP64, cfg.R)
    sysm = oracle_system(cfg.drops)
    b = T(sysm.electric_rhs(cfg.R, cfg.E_u))
    x = torch.empty_like(b)
    it, res = ctx.gmres_solve(S.SYS_ELECTRIC, b, x)
    assert res < 1e-11
    En = sh.sht_inverse(x.cpu().numpy(), 16, 16)
    expect = 3 * cfg.R / (cfg.R + 2) * sysm.drops[0].n0[2]
    assert np.abs(En - expect).max() < 1e-10
    ctx.close()


@pytest.mark.parametrize("system", ["electric", "stokes"])
def test_gmres_two_drops_matches_oracle_solution(S, system):
    cfg = _two_drop_cfg(6, seed=2, gap=0.4)
    sysm = oracle_system(cfg.drops)
    ctx = make(S, cfg.drops, S.FP64, cfg.R)
    rng = np.random.default_rng(4)
    if system == "electric":
        b = sysm.electric_rhs(cfg.R, cfg.E_u)
        ref, _ = gmres.gmres(lambda v: sysm.electric_matvec(cfg.R, v), b, tol=1e-13)
        sid = S.SYS_ELECTRIC
    else:
        b = np.concatenate([inputs.random_density(d.p, rng, 3).ravel() for d in cfg.drops])
        ref, _ = gmres.gmres(sysm.stokes_matvec, b, tol=1e-13)
        sid = S.SYS_STOKES
    x = torch.empty(b.size, device=DEV, dtype=torch.float64)
    it, res = ctx.gmres_solve(sid, T(b), x)
    assert res < 1e-11
    assert rel_err(x.cpu().numpy(), ref) < 1e-9
    ctx.close()


def test_gmres_restart_and_warm_start(S):
    """A small Krylov space forces restarts; a warm start at the solution converges at once."""
    cfg = _two_drop_cfg(5, seed=3, gap=0.4)
    sysm = oracle_system(cfg.drops)
    ctx = S.Context(precision=S.FP64, R=cfg.R, gmres_tol=1e-12, gmres_restart=3)
    ctx.set_drops([d.p for d in cfg.drops], T(np.concatenate([d.xcoef.ravel() for d in cfg.drops])),
                  [d.lam for d in cfg.drops])
    b = sysm.electric_rhs(cfg.R, cfg.E_u)
    x = torch.empty(b.size, device=DEV, dtype=torch.float64)
    it, res = ctx.gmres_solve(S.SYS_ELECTRIC, T(b), x)
    assert res < 1e-11 and it > 3
    it2, res2 = ctx.gmres_solve(S.SYS_ELECTRIC, T(b), torch.empty_like(x), x0=x)
    assert it2 <= 1 and res2 < 1e-11
    ctx.close()


def _spread_drops(rng, nd, p, box=2.6, min_dist=2.35):
    """nd perturbed unit drops of degree p, centres rejection-sampled in [-box, box]^3 at least min_dist
    apart, viscosity ratios U(0.5, 10)."""
    centres = []
    while len(centres) < nd:
        c = rng.uniform(-box, box, 3)
        if all(np.linalg.norm(c - d) > min_dist for d in centres):
            centres.append(c)
    return [inputs.Drop(p, inputs.perturbed_coef(p, rng, 1.0, c), np.zeros(sh.ncoef(p)), float(rng.uniform(0.5, 10.0)),
                        np.asarray(c), 1.0) for c in centres]


def test_stokes_preconditioner_keeps_the_solution_and_cuts_iterations(S):
    """The right preconditioner of the Stokes system (rigid motions and normal mode per drop,
    shbim_set_stokes_preconditioner) on eight drops of viscosity ratios U(0.5, 10): plain and
    preconditioned GMRES reach the oracle's solution, the preconditioned one in at most 3/4 of the
    steps; a warm start, a small Krylov space (restarts every 4 steps) and the mixed-precision refined
    solve keep the solution."""
    rng = np.random.default_rng(12)
    drops = _spread_drops(rng, 8, 5)
    sysm = oracle_system(drops, near=False)
    b = np.concatenate([inputs.random_density(d.p, rng, 3).ravel() for d in drops])
    ref, info = gmres.gmres(sysm.stokes_matvec, b, tol=1e-13)
    its = {}
    for prec in (False, True):
        ctx = make(S, drops, S.FP64, near=False)
        ctx.set_stokes_preconditioner(prec)
        x = torch.empty(b.size, device=DEV, dtype=torch.float64)
        it, res = ctx.gmres_solve(S.SYS_STOKES, T(b), x)
        assert res < 1e-11
        assert rel_err(x.cpu().numpy(), ref) < 1e-9
        its[prec] = it
        if prec:
            # warm start from a perturbed solution
            x0 = T(ref * (1.0 + 1e-3 * rng.standard_normal(ref.size)))
            it2, res2 = ctx.gmres_solve(S.SYS_STOKES, T(b), x, x0=x0)
            assert res2 < 1e-11 and it2 < it
            assert rel_err(x.cpu().numpy(), ref) < 1e-9
            ctx.close()
            # restarts every 4 steps
            ctx = S.Context(precision=S.FP64, R=2.0, gmres_tol=1e-11, gmres_restart=4)
            ctx.set_near(False)
            ctx.set_drops([d.p for d in drops], T(np.concatenate([d.xcoef.ravel() for d in drops])),
                          [d.lam for d in drops])
            it3, res3 = ctx.gmres_solve(S.SYS_STOKES, T(b), x)
            assert res3 < 1e-11
            assert rel_err(x.cpu().numpy(), ref) < 1e-9
            ctx.close()
            # refined mixed-precision solve (FP32 inner solves in one Krylov space)
            ctx = make(S, drops, S.FP32_COMP, near=False)
            inner, outer, r = ctx.gmres_solve_refined(S.SYS_STOKES, T(b), x, inner_tol=1e-5)
            assert r < 1e-8
            assert rel_err(x.cpu().numpy(), ref) < 1e-7
        ctx.close()
    assert its[True] <= 0.75 * its[False], its


@pytest.mark.parametrize("restart", [50, 4])
def test_device_cycles_match_host_steps(S, restart):
    """GMRES with the convergence control on the device (one graph per cycle, a conditional while node
    around the Arnoldi step) against every step on the host: the electric, Stokes and diffusion systems,
    with and without restarts (Krylov dimension 4 forces several cycles); the same number of steps and
    the same solution up to rounding, and the oracle's solution."""
    cfg = _two_drop_cfg(6, seed=7, gap=0.3)
    sysm = oracle_system(cfg.drops)
    rng = np.random.default_rng(8)
    nc = sum(sh.ncoef(d.p) for d in cfg.drops)
    b_e = sysm.electric_rhs(cfg.R, cfg.E_u)
    b_s = rng.standard_normal(3 * nc)
    b_d = rng.standard_normal(nc)
    res = {}
    for device in (True, False):
        ctx = S.Context(precision=S.FP64, R=cfg.R, gmres_tol=1e-11, gmres_restart=restart)
        ctx.set_device_gmres(device)
        ctx.set_drops([d.p for d in cfg.drops], T(np.concatenate([d.xcoef.ravel() for d in cfg.drops])),
                      [d.lam for d in cfg.drops])
        ctx.set_diffusion(0.05)
        out = {}
        for name, sys_, b in (("electric", S.SYS_ELECTRIC, b_e), ("stokes", S.SYS_STOKES, b_s),
                              ("diffusion", S.SYS_DIFFUSION, b_d)):
            x = torch.empty(b.size, device=DEV, dtype=torch.float64)
            for rep in range(2):      # the second solve reuses the cycle graph of the first
                it, r = ctx.gmres_solve(sys_, T(b), x)
                assert r < 1e-10, (device, name, r)
            out[name] = (it, x.cpu().numpy())
        res[device] = out
        ctx.close()
    for name in ("electric", "stokes", "diffusion"):
        it_d, x_d = res[True][name]
        it_h, x_h = res[False][name]
        assert abs(it_d - it_h) <= 1, (name, it_d, it_h)
        assert rel_err(x_d, x_h) < 1e-9, name
    x_ref, _ = gmres.gmres(lambda v: sysm.electric_matvec(cfg.R, v), b_e, tol=1e-13)
    assert rel_err(res[True]["electric"][1], x_ref) < 1e-9


def test_errors_are_reported_not_raised_by_the_library(S):
    ctx = S.Context()
    with pytest.raises(S.ShbimError, match="no drops"):
        ctx.eval_electric(S.LAPLACE_DL, T(np.zeros(4)), T(np.zeros(4)))
    cfg = inputs.config1(3)
    ctx.set_drops([3], T(cfg.drops[0].xcoef.ravel()))
    with pytest.raises(S.ShbimError, match="bad kernel"):
        ctx.eval_electric(7, T(np.zeros(16)), T(np.zeros(16)))
    with pytest.raises(S.ShbimError, match="drop index"):
        ctx.sht(S.SHT_INVERSE, S.GRID_BASE, [2], T(np.zeros(16)), T(np.zeros(32)))
    ctx.close()


@pytest.mark.parametrize("outer", ["df64", "fp64"])
@pytest.mark.parametrize("system", ["electric", "stokes"])
def test_refined_mixed_precision_solve_reaches_fp64_residual(S, system, outer):
    """Iterative refinement: FP32 compensated inner GMRES, FP64-class outer residual (double-
    float or native FP64); the result satisfies the system to 1e-10 and equals the oracle's
    GMRES solution."""
    cfg = _two_drop_cfg(8, seed=5, gap=0.2)
    sysm = oracle_system(cfg.drops)
    rng = np.random.default_rng(8)
    if system == "electric":
        b = sysm.electric_rhs(cfg.R, cfg.E_u)
        ref, _ = gmres.gmres(lambda v: sysm.electric_matvec(cfg.R, v), b, tol=1e-13)
        sid = S.SYS_ELECTRIC
    else:
        b = np.concatenate([inputs.random_density(d.p, rng, 3).ravel() for d in cfg.drops])
        ref, _ = gmres.gmres(sysm.stokes_matvec, b, tol=1e-13)
        sid = S.SYS_STOKES
    ctx = S.Context(precision=S.FP32_COMP, R=cfg.R, gmres_tol=1e-10)
    ctx.set_outer_precision(S.DF64 if outer == "df64" else S.FP64)
    ctx.set_drops([d.p for d in cfg.drops], T(np.concatenate([d.xcoef.ravel() for d in cfg.drops])),
                  [d.lam for d in cfg.drops])
    x = torch.empty(b.size, device=DEV, dtype=torch.float64)
    inner, n_outer, res = ctx.gmres_solve_refined(sid, T(b), x, inner_tol=1e-5, max_outer=8)
    assert res <= 1e-10 and 1 <= n_outer <= 4, (inner, n_outer, res)
    assert rel_err(x.cpu().numpy(), ref) < 1e-9
    ctx.close()


def test_near_pairs_and_corrected_operators_match_oracle(S):
    """Two drops 0.1 apart at p = 8: the library finds the oracle's near pairs and its corrected
    Laplace and Stokes operators (upsampled rule at near targets) match the oracle's."""
    cfg = inputs.config2(p=8, seed=0, gap=0.1)
    cfg.drops[1].lam = 3.0
    sysm = oracle_system(cfg.drops)
    rng = np.random.default_rng(5)
    sig = [inputs.random_density(8, rng, decay=2.0)[0] for _ in cfg.drops]
    f = [inputs.random_density(8, rng, 3, decay=2.0) for _ in cfg.drops]
    nt = 2 * 9 * 18
    ref_l = {kind: np.concatenate(sysm.laplace_grid(kind, sig)) for kind in ("ladl", "lsl")}
    ref_s = np.concatenate([a.ravel() for a in sysm.stokes_grid(f, f)])
    for precision, tol in ((S.FP64, TOL64), (S.DF64, TOL64), (S.FP32_COMP, TOL32)):
        ctx = make(S, cfg.drops, precision, cfg.R)
        assert ctx.near_pairs() == len(sysm.near_pairs()) > 0
        for which, kind in ((S.LAPLACE_DL, "ladl"), (S.LAPLACE_SL, "lsl")):
            out = torch.empty(nt, device=DEV, dtype=torch.float64)
            ctx.eval_electric(which, T(np.concatenate(sig)), out, S.OUT_GRID)
            assert rel_err(out.cpu().numpy(), ref_l[kind]) < tol, (precision, kind)
        out = torch.empty(3 * nt, device=DEV, dtype=torch.float64)
        F = T(np.concatenate([a.ravel() for a in f]))
        ctx.eval_stokes(F, F, out, S.OUT_GRID)
        assert rel_err(out.cpu().numpy(), ref_s) < tol, precision
        ctx.close()
    # without the correction the operators differ from the corrected oracle
    ctx = make(S, cfg.drops, S.FP64, cfg.R, near=False)
    assert ctx.near_pairs() == 0
    out = torch.empty(nt, device=DEV, dtype=torch.float64)
    ctx.eval_electric(S.LAPLACE_DL, T(np.concatenate(sig)), out, S.OUT_GRID)
    assert rel_err(out.cpu().numpy(), np.concatenate(sysm.laplace_grid("ladl", sig))) > 1e-8
    ctx.close()


def test_graph_replay_matches_direct_launches(S):
    """GMRES with its operator applications replayed from CUDA graphs gives the solutions of
    direct launches, in both precisions, and across a change of geometry."""
    cfg = _two_drop_cfg(8, seed=6, gap=0.2)
    rng = np.random.default_rng(9)
    b_s = T(np.concatenate([inputs.random_density(8, rng, 3).ravel() for _ in cfg.drops]))
    out = {}
    for graphs in (False, True):
        for precision in (S.FP64, S.FP32_COMP, S.DF64):
            ctx = S.Context(precision=precision, R=cfg.R, gmres_tol=1e-10)
            ctx.set_graphs(graphs)
            ctx.set_autotune(False)     # the same FP32 summation order in both contexts
            sols = []
            for shift in (0.0, 0.05):
                xc = np.concatenate([d.xcoef.ravel() for d in cfg.drops])
                xc[0] += shift          # moves drop 0 in x: a new geometry, graphs re-captured
                ctx.set_drops([d.p for d in cfg.drops], T(xc), [d.lam for d in cfg.drops])
                nc = b_s.numel() // 3
                rhs = torch.empty(nc, device=DEV, dtype=torch.float64)
                ctx.electric_rhs(cfg.E_u, rhs)
                xe = torch.empty_like(rhs)
                ie, _ = ctx.gmres_solve(S.SYS_ELECTRIC, rhs, xe)
                xs = torch.empty_like(b_s)
                is_, _ = ctx.gmres_solve(S.SYS_STOKES, b_s, xs)
                sols.append((ie, is_, xe.cpu().numpy(), xs.cpu().numpy()))
            out[(graphs, precision)] = sols
            ctx.close()
    for precision in (S.FP64, S.FP32_COMP, S.DF64):
        for a, b in zip(out[(False, precision)], out[(True, precision)]):
            assert a[0] == b[0] and a[1] == b[1]
            assert rel_err(b[2], a[2]) < 1e-10 and rel_err(b[3], a[3]) < 1e-10


def test_concurrent_branches_match_serial_order(S):
    """Two drops 0.1 apart (near pairs exist): with the self rows and the near-field correction
    on the library's second stream, every operator and a graph-replayed GMRES solve give the
    serial results up to the rounding of the changed summation order."""
    cfg = _two_drop_cfg(8, seed=2, gap=0.1)
    rng = np.random.default_rng(11)
    sig = T(np.concatenate([inputs.random_density(8, rng)[0] for _ in cfg.drops]))
    F = T(np.concatenate([inputs.random_density(8, rng, 3).ravel() for _ in cfg.drops]))
    for precision in (S.FP64, S.FP32_COMP, S.DF64):
        res = {}
        for conc in (False, True):
            ctx = make(S, cfg.drops, precision, cfg.R)
            assert ctx.near_pairs() > 0
            ctx.set_autotune(False)
            ctx.set_concurrency(conc)
            outs = []
            for which in (S.LAPLACE_DL, S.LAPLACE_SL):
                out = torch.empty(sig.numel(), device=DEV, dtype=torch.float64)
                ctx.eval_electric(which, sig, out, S.OUT_COEF)
                outs.append(out.cpu().numpy())
            for f, u in ((F, None), (None, F), (F, F)):
                out = torch.empty(F.numel(), device=DEV, dtype=torch.float64)
                ctx.eval_stokes(f, u, out, S.OUT_COEF)
                outs.append(out.cpu().numpy())
            ctx.close()
            # GMRES with graph replay of the forked application (FP32: to its own accuracy)
            ctx = S.Context(precision=precision, R=cfg.R, gmres_tol=1e-5 if precision == S.FP32_COMP else 1e-10)
            ctx.set_autotune(False)
            ctx.set_concurrency(conc)
            ctx.set_drops([d.p for d in cfg.drops], T(np.concatenate([d.xcoef.ravel() for d in cfg.drops])),
                          [d.lam for d in cfg.drops])
            xs = torch.empty_like(F)
            its, _ = ctx.gmres_solve(S.SYS_STOKES, F, xs)
            outs.append(xs.cpu().numpy())
            res[conc] = (outs, its)
            ctx.close()
        assert res[False][1] == res[True][1], precision
        for a, b in zip(res[False][0], res[True][0]):
            assert rel_err(b, a) < 1e-12, precision


def test_two_lane_row_build_gives_the_same_rows(S):
    """The double-float row build with every other chunk of targets on the library's second
    stream gives the serial build's rows bit for bit (compared through serial operator
    applications without the near-field atomics)."""
    cfg = _two_drop_cfg(9, seed=4, gap=0.3)
    rng = np.random.default_rng(13)
    sig = T(np.concatenate([inputs.random_density(9, rng)[0] for _ in cfg.drops]))
    F = T(np.concatenate([inputs.random_density(9, rng, 3).ravel() for _ in cfg.drops]))
    outs = {}
    for lanes in (True, False):
        ctx = S.Context(precision=S.FP64, R=cfg.R, gmres_tol=1e-12)
        ctx.set_near(False)
        ctx.set_concurrency(lanes)
        ctx.set_drops([d.p for d in cfg.drops], T(np.concatenate([d.xcoef.ravel() for d in cfg.drops])),
                      [d.lam for d in cfg.drops])
        ctx.set_concurrency(False)          # serial applications: a fixed summation order
        res = []
        for which in (S.LAPLACE_DL, S.LAPLACE_SL):
            out = torch.empty(sig.numel(), device=DEV, dtype=torch.float64)
            ctx.eval_electric(which, sig, out, S.OUT_COEF)
            res.append(out.cpu().numpy())
        out = torch.empty(F.numel(), device=DEV, dtype=torch.float64)
        ctx.eval_stokes(F, F, out, S.OUT_COEF)
        res.append(out.cpu().numpy())
        outs[lanes] = res
        ctx.close()
    for a, b in zip(outs[True], outs[False]):
        assert np.array_equal(a, b)
