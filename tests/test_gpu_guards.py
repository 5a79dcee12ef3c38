"""Bounded waits and the closest-approach guard of the nearly-singular rule, through the C ABI.

* A wait inside a kernel runs out after the context's limit and the call returns
  SHBIM_ERR_TIMEOUT, with the context still usable (shbim_check_wait waits on a barrier that
  nothing arrives on; no copy or product is in flight meanwhile).
* shbim_set_drops measures the smallest distance from a near target to another drop's surface,
  sampled on that drop's four-times upsampled grid; the oracle's geometry gives the same minimum.
"""
import math
import os
import time

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = torch.device("cuda")


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


def test_bounded_wait_runs_out_and_the_context_stays_usable(S):
    ctx = S.Context()
    assert ctx.check_wait(arrive=True) == 0
    ctx.set_wait_limit(0.05)
    t0 = time.perf_counter()
    assert ctx.check_wait(arrive=False) == S.ERR_TIMEOUT
    assert time.perf_counter() - t0 >= 0.05
    # the device and the context are fine afterwards
    assert ctx.check_wait(arrive=True) == 0
    cfg = inputs.config1(4)
    ctx.set_drops([4], torch.tensor(cfg.drops[0].xcoef.ravel(), device=DEV))
    out = torch.empty(25, device=DEV, dtype=torch.float64)
    ctx.eval_electric(S.LAPLACE_SL, torch.tensor(np.eye(25)[0], device=DEV), out)
    torch.cuda.synchronize()
    assert np.isfinite(out.cpu().numpy()).all()
    with pytest.raises(S.ShbimError, match="wait limit"):
        ctx.set_wait_limit(0.0)
    ctx.close()


@pytest.mark.parametrize("p,gap", [(8, 0.1), (12, 0.05)])
def test_closest_approach_matches_oracle(S, p, gap):
    from oracle import geometry, nearsing, operators
    cfg = inputs.config2(p=p, seed=0, gap=gap)
    ctx = S.Context(precision=S.FP64, R=cfg.R)
    ctx.set_drops([p, p], torch.tensor(np.concatenate([d.xcoef.ravel() for d in cfg.drops]), device=DEV))
    dist, ratio = ctx.near_min_distance()
    ctx.close()
    sysm = operators.System([operators.DropGeom(d.xcoef, d.p, d.lam) for d in cfg.drops])
    best, best_r = math.inf, math.inf
    for (i, t, j) in nearsing.near_pairs(sysm):
        dj = sysm.drops[j]
        xf, _, _ = geometry.surface_on_grid(dj.xcoef, dj.p, nearsing.near_degree(dj))
        d = math.sqrt(((xf - sysm.drops[i].x0[:, t:t + 1]) ** 2).sum(0).min())
        best = min(best, d)
        best_r = min(best_r, d / nearsing.spacing(dj))
    assert math.isfinite(best)
    assert abs(dist - best) < 1e-5 * best + 1e-6
    assert abs(ratio - best_r) < 1e-5 * best_r + 1e-6
    assert ratio < 6.0


def test_closest_approach_is_infinite_without_near_pairs(S):
    p = 6
    x0 = inputs.sphere_coef(p, 1.0, (0.0, 0.0, 0.0))
    x1 = inputs.sphere_coef(p, 1.0, (0.0, 0.0, 5.0))
    ctx = S.Context(precision=S.FP64)
    ctx.set_drops([p, p], torch.tensor(np.concatenate([x0.ravel(), x1.ravel()]), device=DEV))
    assert ctx.near_pairs() == 0
    assert ctx.near_min_distance() == (math.inf, math.inf)
    ctx.close()
