"""The seeded two-drop and batched inputs keep the surface gap the generator promises.

The generator draws the shape perturbations without looking at the surfaces (it holds none of the
method's arithmetic), so the gap of every seed that the tests and the benchmark use is checked here, by
the oracle's geometry on a fine grid: the smallest distance between two drops' surfaces must be at
least half the nominal gap (seeds that fail would be redrawn as seed + 1000 k)."""
import math

import numpy as np
import pytest

import inputs
from oracle import geometry


def _closest(da, db, q, xa=None, xb=None):
    if xa is None:
        xa, _, _ = geometry.surface_on_grid(da.xcoef, da.p, q)
    if xb is None:
        xb, _, _ = geometry.surface_on_grid(db.xcoef, db.p, q)
    # only the caps facing each other can hold the closest pair
    ca = np.asarray(da.centre, float)
    cb = np.asarray(db.centre, float)
    axis = (cb - ca) / np.linalg.norm(cb - ca)
    sa = xa[:, ((xa - ca[:, None]) * axis[:, None]).sum(0) > 0.5 * da.radius]
    sb = xb[:, ((xb - cb[:, None]) * axis[:, None]).sum(0) < -0.5 * db.radius]
    best = math.inf
    for k in range(0, sa.shape[1], 512):
        d = sa[:, k:k + 512, None] - sb[:, None, :]
        best = min(best, float(np.sqrt((d * d).sum(0)).min()))
    return best


@pytest.mark.parametrize("p,seed,gap", [(32, 0, 0.1), (8, 0, 0.1), (12, 2, 0.1), (12, 0, 0.05), (8, 1, 0.1)])
def test_two_drop_seeds_keep_half_the_nominal_gap(p, seed, gap):
    cfg = inputs.config2(p=p, seed=seed, gap=gap)
    d = _closest(cfg.drops[0], cfg.drops[1], 2 * p + 1)
    assert d >= 0.5 * gap, (p, seed, gap, d)


def test_batched_seed_keeps_half_the_minimum_gap():
    cfg = inputs.config3(seed=3)
    surf = {}

    def x_of(k):
        if k not in surf:
            d = cfg.drops[k]
            surf[k] = geometry.surface_on_grid(d.xcoef, d.p, d.p + 8)[0]
        return surf[k]
    worst = math.inf
    for i, a in enumerate(cfg.drops):
        for j in range(i + 1, len(cfg.drops)):
            b = cfg.drops[j]
            centre_gap = np.linalg.norm(np.asarray(a.centre) - np.asarray(b.centre)) - a.radius - b.radius
            if centre_gap < 0.6:     # nominal gap >= 0.4 (0.2 + 0.2 slack): only close pairs need a look
                worst = min(worst, _closest(a, b, None, x_of(i), x_of(j)))
    assert worst >= 0.1, worst
