"""The reparametrisation kernels (Section 2.2, after every accepted step of Algorithm 1) against the
oracle: positions, carried concentration and energies, drop by drop."""
import os

import numpy as np
import pytest

import inputs
from oracle import reparam

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


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


def _run(S, drops, steps, a=4.0, c=0.5, gamma=True):
    x = torch.tensor(np.concatenate([d.xcoef.ravel() for d in drops]), device="cuda")
    g = torch.tensor(np.concatenate([d.gamma_coef for d in drops]), device="cuda") if gamma else None
    ctx = S.Context(precision=S.FP64)
    ctx.set_drops([d.p for d in drops], x, [d.lam for d in drops])
    e = ctx.reparametrize(x, g, steps=steps, a=a, c=c)
    ctx.close()
    return x.cpu().numpy(), (g.cpu().numpy() if gamma else None), np.array(e)


def _split(v, drops, per):
    out, o = [], 0
    for d in drops:
        n = per * inputs.ncoef(d.p)
        out.append(v[o:o + n].reshape(per, -1) if per > 1 else v[o:o + n])
        o += n
    return out


def _check(drops, x, g, e, steps, a, c, which=None):
    xs, gs = _split(x, drops, 3), (_split(g, drops, 1) if g is not None else None)
    e_ref = 0.0
    which = range(len(drops)) if which is None else which
    for i in which:
        d = drops[i]
        if g is None:
            xr, hist = reparam.reparametrize(d.xcoef, d.p, steps=steps, a=a, c=c)
        else:
            xr, hist, gr = reparam.reparametrize(d.xcoef, d.p, steps=steps, a=a, c=c, gamma=d.gamma_coef)
            assert np.abs(gs[i] - gr).max() <= 1e-11 * np.abs(gr).max(), i
        assert np.abs(xs[i] - xr).max() <= 1e-11 * np.abs(xr).max(), i
        e_ref = e_ref + np.array(hist)
    return e_ref


def test_mixed_degrees_match_oracle(S):
    """Three drops, two of degree 6 (one launch per degree group) and one of degree 9 (grids of 14 and 20
    latitudes: ragged 128-node tiles); 6 steps with the concentration; energies summed over the drops.
    FP64 on both sides: tolerance 1e-11 of the largest coefficient (different summation orders)."""
    rng = np.random.default_rng(21)
    drops = []
    for p, ctr in ((6, (0, 0, 0)), (9, (3, 0, 0)), (6, (0, 3.2, 0))):
        drops.append(inputs.Drop(p=p, xcoef=inputs.perturbed_coef(p, rng, 1.0, ctr),
                                 gamma_coef=inputs.gamma_random(p, rng), lam=1.0,
                                 centre=np.asarray(ctr, float), radius=1.0))
    x, g, e = _run(S, drops, 6, a=4.0, c=0.5)
    e_ref = _check(drops, x, g, e, 6, 4.0, 0.5)
    np.testing.assert_allclose(e, e_ref, rtol=1e-12)
    assert np.all(np.diff(e) < 0)
    # another exponent and step factor, positions only
    x, _, e = _run(S, drops, 3, a=2.0, c=1.0, gamma=False)
    np.testing.assert_allclose(e, _check(drops, x, None, e, 3, 2.0, 1.0), rtol=1e-12)


def test_zero_steps_reports_energy_only(S):
    rng = np.random.default_rng(4)
    d = inputs.Drop(p=8, xcoef=inputs.perturbed_coef(8, rng, 1.0, (0, 0, 0)), gamma_coef=inputs.gamma_random(8, rng),
                    lam=1.0, centre=np.zeros(3), radius=1.0)
    x, g, e = _run(S, [d], 0)
    assert np.array_equal(x, d.xcoef.ravel()) and np.array_equal(g, d.gamma_coef)
    assert len(e) == 1 and abs(e[0] - reparam.energy(d.xcoef, 8)) <= 1e-13 * e[0]


def test_batched_workload_sampled_drops(S):
    """The batched workload (64 drops of degree 16-48, the time step's layout): two steps with the
    concentration, checked against the oracle on one drop of each degree."""
    cfg = inputs.config3()
    drops = cfg.drops
    sample = []
    for p in sorted({d.p for d in drops}):
        sample.append(next(i for i, d in enumerate(drops) if d.p == p))
    x, g, e = _run(S, drops, 2)
    _check(drops, x, g, e, 2, 4.0, 0.5, which=sample)
    e_all = sum(reparam.energy(d.xcoef, d.p) for d in drops)
    assert abs(e[0] - e_all) <= 1e-12 * e_all and e[2] < e[0]


def test_arguments_are_checked(S):
    d = inputs.Drop(p=4, xcoef=inputs.sphere_coef(4), gamma_coef=np.zeros(25), lam=1.0, centre=np.zeros(3), radius=1.0)
    x = torch.tensor(d.xcoef.ravel(), device="cuda")
    ctx = S.Context(precision=S.FP64)
    ctx.set_drops([4], x, [1.0])
    for kw in ({"c": 0.0}, {"c": 1.5}, {"a": -1.0}, {"a": 9.0}, {"steps": -1}):
        with pytest.raises(S.ShbimError):
            ctx.reparametrize(x, None, **kw)
    with pytest.raises(S.ShbimError):
        ctx.reparametrize(x, x[10:35], steps=1)            # concentration overlapping the positions
    ctx.close()
