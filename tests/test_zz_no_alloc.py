"""The allocation-free Laplace pair sum against the FP64 oracle and the library's operator entry point.

shbim_pairs_laplace_noalloc serves callers that cannot allocate device memory when they call it
(for example a host application that reserves all of its device memory up front); it keeps its
partial sums in a fixed array in device memory instead of allocating scratch.

Set-up: two drops far enough apart that no target is near the other drop, drop 1 a sphere of radius
a, whose upsampled-grid nodes and regular weights are known in closed form (J = a^2). The targets
(drop 0's grid, perturbed shape) and the source strengths come from the oracle; the expected sums
are the oracle's regular rule (Eq. reg_quadrature) over the same arrays, and, with the density
zero on drop 0, also the value of shbim_eval_electric at drop 0's targets. Collected last (file
name) so that a run that stops at the first failure has already run every other test.
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
def test_noalloc_pair_sum_matches_oracle_and_operator(S, which):
    from oracle import geometry, quadrature, sh
    p = 10
    a, centre = 0.9, np.array([0.1, -0.2, 3.1])
    rng = np.random.default_rng(21)
    x0 = inputs.perturbed_coef(p, rng, 1.0, (0.0, 0.0, 0.0))
    x1 = inputs.sphere_coef(p, a, centre)
    sig1 = inputs.random_density(p, rng)[0]
    # the oracle's arrays: drop 0's targets and drop 1's quadrature sources
    xt, nt_, _ = geometry.surface_on_grid(x0, p, p)
    xs, w = _sphere_sources(p, a, centre)
    dens = sh.sht_inverse(sig1, p, 2 * p + 1)
    kind = "ladl" if which == 0 else "lsl"
    expect = quadrature.regular_scalar(kind, xt, nt_, xs, w, dens)
    dev = torch.device("cuda")
    tgt = torch.tensor(np.concatenate([xt, nt_]), device=dev).contiguous()
    src = torch.tensor(np.concatenate([xs, (dens * w)[None]]), device=dev).contiguous()
    nt = xt.shape[1]
    # the library's own operator on the same layout (drop 1's density only)
    ctx = S.Context(precision=S.FP64)
    ctx.set_drops([p, p], torch.tensor(np.concatenate([x0.ravel(), x1.ravel()]), device=dev))
    assert ctx.near_pairs() == 0     # far apart: the operator is the plain regular sum
    nc = (p + 1) ** 2
    ref = torch.empty(2 * nt, device=dev, dtype=torch.float64)
    ctx.eval_electric(which, torch.tensor(np.concatenate([np.zeros(nc), sig1]), device=dev), ref, S.OUT_GRID)
    op = ref[:nt].cpu().numpy()
    ctx.close()
    torch.cuda.synchronize()
    for call in range(2):
        out = torch.full((nt,), float("nan"), device=dev, dtype=torch.float64)
        torch.cuda.synchronize()
        alloc0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
        rc = S.pairs_laplace_noalloc(which, tgt, src, out)
        torch.cuda.synchronize()
        assert rc == 0
        if call == 1:   # the first call may load the module's code; later calls take no memory
            assert torch.cuda.memory_allocated() == alloc0
            assert torch.cuda.mem_get_info()[0] == free0
        got = out.cpu().numpy()
        for ref_ in (expect, op):
            err = max(np.linalg.norm(got - ref_) / np.linalg.norm(ref_),
                      np.abs(got - ref_).max() / np.abs(ref_).max())
            assert err < 1e-10, (call, err)


def test_noalloc_rejects_sizes_beyond_its_scratch(S):
    import ctypes
    dev = torch.device("cuda")
    t = torch.zeros(6, device=dev, dtype=torch.float64)
    s = torch.zeros(4, device=dev, dtype=torch.float64)
    o = torch.zeros(1, device=dev, dtype=torch.float64)
    raw = S.lib().shbim_pairs_laplace_noalloc
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda x: ctypes.c_void_p(x.data_ptr())   # noqa: E731
    # the size check comes before any device work, so the oversize count never reaches a kernel
    assert raw(0, ptr(t), S.NOALLOC_MAX_TARGETS + 1, ptr(s), 1, ptr(o), st) == S.ERR_ARG
    assert raw(5, ptr(t), 1, ptr(s), 1, ptr(o), st) == S.ERR_ARG
    # the binding refuses tensors smaller than the counts it would pass
    with pytest.raises(S.ShbimError):
        S.pairs_laplace_noalloc(0, t, s, torch.zeros(2, device=dev, dtype=torch.float64))
