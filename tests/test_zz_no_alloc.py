"""The allocation-free Laplace pair sum, checked against the library's operator entry point.

shbim_pairs_laplace_noalloc serves callers that must not allocate device memory while they
run (for example code that executes inside a CUDA stream capture, or inside a host process
whose device memory is budgeted up front); it keeps its partial sums in a fixed array in
device memory instead of allocating scratch.

Set-up: two drops far enough apart that no target is near the other drop, drop 1 a sphere of radius a, whose upsampled-grid nodes and regular
weights are known in closed form (J = a^2). With the density zero on drop 0, the value of
shbim_eval_electric at drop 0's targets is exactly the regular sum over drop 1's sources, which
is what the allocation-free call computes from explicit arrays. Collected last (file name) so
that a run that stops at the first failure has already run every other test.
"""
import math
import os

import numpy as np
import pytest

import inputs

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


def _sphere_sources(p, a, centre):
    q = 2 * p + 1
    x, w = np.polynomial.legendre.leggauss(q + 1)
    t, wg = x[::-1], w[::-1]
    th = np.arccos(t)
    ph = np.pi * np.arange(2 * q + 2) / (q + 1)
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    X = centre[0] + a * np.sin(TH) * np.cos(PH)
    Y = centre[1] + a * np.sin(TH) * np.sin(PH)
    Z = centre[2] + a * np.cos(TH)
    W = np.repeat(np.pi / (q + 1) * wg * a * a, 2 * q + 2)
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()]), W


@pytest.mark.parametrize("which", [0, 1])
def test_noalloc_pair_sum_matches_operator_entry_point(S, which):
    p = 10
    a, centre = 0.9, np.array([0.1, -0.2, 3.1])
    rng = np.random.default_rng(21)
    x0 = inputs.perturbed_coef(p, rng, 1.0, (0.0, 0.0, 0.0))
    x1 = inputs.sphere_coef(p, a, centre)
    dev = torch.device("cuda")
    ctx = S.Context(precision=S.FP64)
    ctx.set_drops([p, p], torch.tensor(np.concatenate([x0.ravel(), x1.ravel()]), device=dev))
    assert ctx.near_pairs() == 0     # far apart: the operator is the plain regular sum
    nc = (p + 1) ** 2
    nt = (p + 1) * (2 * p + 2)
    sig1 = inputs.random_density(p, rng)[0]
    sig = torch.tensor(np.concatenate([np.zeros(nc), sig1]), device=dev)
    ref = torch.empty(2 * nt, device=dev, dtype=torch.float64)
    ctx.eval_electric(which, sig, ref, S.OUT_GRID)
    geo = torch.empty(7 * 2 * nt, device=dev, dtype=torch.float64)
    ctx.target_geometry(geo)
    geo = geo.view(7, 2 * nt)
    tgt = geo[:6, :nt].contiguous()
    xs, w = _sphere_sources(p, a, centre)
    ns = xs.shape[1]
    sig_up = torch.empty(ns, device=dev, dtype=torch.float64)
    ctx.sht(1, S.SHT_INVERSE, S.GRID_UP, 1, torch.tensor(sig1, device=dev), sig_up)
    src = torch.cat([torch.tensor(xs, device=dev), (sig_up * torch.tensor(w, device=dev))[None]]).contiguous()
    expect = ref[:nt].cpu().numpy()
    for _ in range(2):
        out = torch.full((nt,), float("nan"), device=dev, dtype=torch.float64)
        rc = S.pairs_laplace_noalloc(which, tgt, src, out)
        assert rc == 0
        got = out.cpu().numpy()
        err = max(np.linalg.norm(got - expect) / np.linalg.norm(expect),
                  np.abs(got - expect).max() / np.abs(expect).max())
        assert err < 1e-10, err
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(S):
    dev = torch.device("cuda")
    t = torch.zeros(6, device=dev, dtype=torch.float64)
    s = torch.zeros(4, device=dev, dtype=torch.float64)
    o = torch.zeros(1, device=dev, dtype=torch.float64)
    assert S.pairs_laplace_noalloc(0, t, s, o, n_tgt=S.NOALLOC_MAX_TARGETS + 1, n_src=1) == -1
    assert S.pairs_laplace_noalloc(5, t, s, o, n_tgt=1, n_src=1) == -1
