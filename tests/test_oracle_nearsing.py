"""Pins of the oracle's nearly-singular correction (Section 2.1): at targets close to another
drop, the corrected value equals brute force -- the regular rule with the sources upsampled
sixteen times per direction -- while the plain degree-q rule does not."""
import math

import numpy as np
import pytest

import inputs
from oracle import geometry, nearsing, operators, quadrature, sh


@pytest.fixture(scope="module")
def close_pair():
    cfg = inputs.config2(p=8, seed=0, gap=0.1)
    cfg.drops[1].lam = 3.0
    drops = [operators.DropGeom(d.xcoef, d.p, d.lam) for d in cfg.drops]
    return operators.System(drops, near=True), drops


def test_near_pairs_are_the_targets_within_six_spacings(close_pair):
    sysm, drops = close_pair
    pairs = sysm.near_pairs()
    assert len(pairs) > 10
    for (i, t, j) in pairs:
        d = drops[j].xs - drops[i].x0[:, t:t + 1]
        assert math.sqrt((d * d).sum(0).min()) < 6 * nearsing.spacing(drops[j])
    # the far sides of the drops are not near
    far = [t for t in range(drops[0].nt) if drops[0].x0[2, t] < -1.5]
    assert far and not any(t in far for (i, t, j) in pairs if i == 0)


def test_near_pairs_of_one_drop_agree_with_the_full_list(close_pair):
    """near_pairs_of (one drop's targets, bounding-sphere filter) gives that drop's part of near_pairs,
    for all its targets and for a subset."""
    sysm, drops = close_pair
    pairs = sysm.near_pairs()
    for i in range(2):
        mine = sorted(pr for pr in pairs if pr[0] == i)
        assert sorted(nearsing.near_pairs_of(sysm, i)) == mine
        sub = sorted({t for (_, t, _) in mine[::3]} | {0, drops[i].nt - 1})
        assert sorted(nearsing.near_pairs_of(sysm, i, sub)) == sorted(pr for pr in mine if pr[1] in sub)


def _brute(kind, dj, x0, n0, dens_coef):
    qf = 16 * (dj.q + 1) - 1
    x, n, J = geometry.surface_on_grid(dj.xcoef, dj.p, qf)
    w = sh.grid_weights(qf) * J
    if kind in ("lsl", "ladl"):
        return quadrature.regular_scalar(kind, x0, n0, x, w, sh.sht_inverse(dens_coef, dj.p, qf))[0]
    return quadrature.regular_tensor(kind, x0, x, n, w, sh.sht_inverse(dens_coef, dj.p, qf))[:, 0]


def test_corrected_values_match_brute_force(close_pair):
    sysm, drops = close_pair
    rng = np.random.default_rng(5)
    sig = [inputs.random_density(8, rng, decay=2.0)[0] for _ in drops]
    f = [inputs.random_density(8, rng, 3, decay=2.0) for _ in drops]
    pairs = sysm.near_pairs()
    sub = [pr for pr in pairs if pr[0] == 0][::4]
    for kind in ("lsl", "ladl"):
        plain = operators.System(drops).laplace_grid(kind, sig)
        corr = sysm.laplace_grid(kind, sig)
        worst_plain = 0.0
        for (i, t, j) in sub:
            di, dj = drops[i], drops[j]
            x0, n0 = di.x0[:, t:t + 1], di.n0[:, t:t + 1]
            own = corr[i][t] - (plain[i][t] - quadrature.regular_scalar(
                kind, x0, n0, dj.xs, dj.ws, sh.sht_inverse(sig[j], 8, dj.q))[0])
            ref = _brute(kind, dj, x0, n0, sig[j])
            assert abs(own - ref) < 1e-9 * max(1.0, abs(ref))
            worst_plain = max(worst_plain, abs(plain[i][t] - corr[i][t]))
        assert worst_plain > 1e-6          # the correction matters at these targets
    corr = sysm.stokes_grid(f, f)
    plain = operators.System(drops).stokes_grid(f, f)
    for (i, t, j) in sub[:4]:
        di, dj = drops[i], drops[j]
        x0 = di.x0[:, t:t + 1]
        reg = (quadrature.regular_tensor("sto_s", x0, dj.xs, dj.ns, dj.ws, sh.sht_inverse(f[j], 8, dj.q))[:, 0]
               + (dj.lam - 1) * quadrature.regular_tensor("sto_d", x0, dj.xs, dj.ns, dj.ws,
                                                         sh.sht_inverse(f[j], 8, dj.q))[:, 0])
        own = corr[i][:, t] - (plain[i][:, t] - reg)
        ref = _brute("sto_s", dj, x0, None, f[j]) + (dj.lam - 1) * _brute("sto_d", dj, x0, None, f[j])
        assert np.abs(own - ref).max() < 1e-8 * max(1.0, np.abs(ref).max())
