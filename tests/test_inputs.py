"""The seeded input generators: deterministic per seed, and the stated recipe holds (degrees, radii,
viscosity ratios, drops inside the box, nominal gaps, surfaces of the two-drop workload kept apart)."""
import numpy as np

import inputs
from oracle import sh


def test_generators_are_deterministic_per_seed():
    a, b, c = inputs.config2(p=8, seed=3), inputs.config2(p=8, seed=3), inputs.config2(p=8, seed=4)
    for da, db in zip(a.drops, b.drops):
        assert np.array_equal(da.xcoef, db.xcoef) and np.array_equal(da.gamma_coef, db.gamma_coef)
    assert not np.array_equal(a.drops[0].xcoef, c.drops[0].xcoef)


def _nominal_gaps_ok(cfg, gap, box):
    ctr = np.array([d.centre for d in cfg.drops])
    rad = np.array([d.radius for d in cfg.drops])
    assert np.all(np.abs(ctr) + rad[:, None] <= box / 2 + 1e-12)
    dist = np.linalg.norm(ctr[:, None, :] - ctr[None, :, :], axis=-1)
    need = rad[:, None] + rad[None, :] + gap
    np.fill_diagonal(dist, np.inf)
    assert np.all(dist >= need - 1e-12)


def test_batched_workload_recipe():
    cfg = inputs.config3()
    assert len(cfg.drops) == 64
    assert {d.p for d in cfg.drops} <= {16, 24, 32, 48} and len({d.p for d in cfg.drops}) == 4
    assert all(0.8 <= d.radius <= 1.2 and 0.5 <= d.lam <= 10.0 for d in cfg.drops)
    _nominal_gaps_ok(cfg, 0.4, 12.0)


def test_large_workload_recipe():
    cfg = inputs.config5()
    assert len(cfg.drops) == 16 and all(d.p == 64 and d.radius == 1.0 and d.lam == 1.0 for d in cfg.drops)
    assert sum((2 * d.p + 2) * (4 * d.p + 4) for d in cfg.drops) == 540800   # degree 2p+1 source nodes
    _nominal_gaps_ok(cfg, 0.4, 8.0)


def test_two_drop_surfaces_stay_apart():
    """Nominal surface gap 0.1: for the timing seeds the perturbed surfaces, sampled on the degree
    2p+1 grid, stay at least half of it apart, and the surfactant stays within 0.2 of 1."""
    p = 32
    th, ph = sh.grid_points(2 * p + 1)
    Y = sh.basis(p, np.cos(th).ravel(), np.sin(th).ravel(), ph.ravel())
    for seed in range(10):
        cfg = inputs.config2(p=p, seed=seed)
        lo, hi = (d.xcoef @ Y for d in cfg.drops)          # lower drop, upper drop
        A = lo[:, np.argsort(lo[2])[-1500:]].T              # the facing caps
        B = hi[:, np.argsort(hi[2])[:1500]].T
        dmin = np.sqrt(((A[:, None, :] - B[None, :, :]) ** 2).sum(-1)).min()
        assert dmin >= 0.05, (seed, dmin)
        for d in cfg.drops:
            assert np.abs(d.gamma_coef @ Y - 1.0).max() <= 0.2
