"""The warm-start network's kernels against the oracle, and what the trained network gains."""
import os

import numpy as np
import pytest

import inputs
from oracle import mlp as M

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


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_forward_and_gradients_match_oracle(S):
    """Widths that leave ragged 64 x 64 tiles in every product; bfloat16 operands, FP32
    accumulation. Tolerance 2e-2 (relative L2): a bfloat16 rounding carries 2^-9 relative error
    and the backward products round their operands too, which the FP64 oracle does not."""
    widths = [70, 96, 64, 40]
    Ws, bs = M.init(widths, 7)
    rng = np.random.default_rng(2)
    bs = [(b + 0.1 * rng.standard_normal(b.shape)).astype(np.float32) for b in bs]
    x = rng.standard_normal((13, 70)).astype(np.float32)
    t = rng.standard_normal((13, 40)).astype(np.float32)
    net = S.MLP(widths, max_batch=16)
    for l in range(3):
        net.set_layer(l, Ws[l], bs[l])
    X = torch.tensor(x, device="cuda")
    Y = torch.empty((13, 40), device="cuda", dtype=torch.float32)
    net.forward(X, Y)
    hs, _ = M.forward(Ws, bs, x)
    assert rel(Y.cpu().numpy(), hs[-1]) < 1e-2
    loss = net.train_step(X, torch.tensor(t, device="cuda"), 0.0, update=False)
    ref_loss, gW, gb = M.loss_and_grads(Ws, bs, x, t)
    assert abs(loss - ref_loss) < 1e-2 * ref_loss
    for l in range(3):
        _, _, gWd, gbd = net.get_layer(l)
        assert rel(gWd, gW[l]) < 2e-2
        assert rel(gbd, gb[l]) < 2e-2
    net.close()


def test_adam_step_matches_oracle(S):
    widths = [33, 64, 17]
    Ws, bs = M.init(widths, 11)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((8, 33)).astype(np.float32)
    t = rng.standard_normal((8, 17)).astype(np.float32)
    net = S.MLP(widths, max_batch=8)
    for l in range(2):
        net.set_layer(l, Ws[l], bs[l])
    net.train_step(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"), 1e-2, update=True)
    for l in range(2):
        W, b, gW, gb = net.get_layer(l)
        Wr, _, _ = M.adam(Ws[l].astype(np.float64), gW.astype(np.float64), 0.0, 0.0, 1, 1e-2)
        br, _, _ = M.adam(bs[l].astype(np.float64), gb.astype(np.float64), 0.0, 0.0, 1, 1e-2)
        np.testing.assert_allclose(W, Wr, rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(b, br, rtol=1e-5, atol=1e-6)
    net.close()


def test_trained_warm_start_saves_gmres_iterations(S):
    """Train on solves of two-drop inputs made by the method itself (p = 6, 600 seeds) and
    compare, on 16 held-out seeds, three initial guesses: zero, the sphere solution
    3R/(R+2) E.n, and sphere + network. The network must cut the initial relative residual of
    the electric system well below the sphere guess's and never cost GMRES iterations; the
    solutions GMRES reaches from any start agree (GMRES judges the error)."""
    from paper_1811_10270_gb300 import warmstart
    p = 6
    Xtr, Ytr, _ = warmstart.generate(inputs.config2(p=p, seed=sd, gap=0.1) for sd in range(1, 601))
    net, hist = warmstart.train(Xtr, Ytr, hidden=(256, 256, 256), epochs=150, batch=32, lr=1e-3)
    assert hist[-1] < 0.2 * hist[0]
    counts = {"zero": [], "sphere": [], "learned": []}
    r0 = {"sphere": [], "learned": []}
    for sd in range(100000, 100016):
        cfg = inputs.config2(p=p, seed=sd, gap=0.1)
        ctx = S.Context(precision=S.FP64, R=cfg.R, gmres_tol=1e-10)
        x = torch.tensor(np.concatenate([d.xcoef.ravel() for d in cfg.drops]), device="cuda")
        ctx.set_drops([p, p], x, [d.lam for d in cfg.drops])
        nc = x.numel() // 3
        rhs = torch.empty(nc, device="cuda", dtype=torch.float64)
        ctx.electric_rhs(cfg.E_u, rhs)
        sols = {}
        for name in counts:
            if name == "zero":
                x0 = None
            elif name == "sphere":
                x0 = 3.0 * (cfg.R + 1) / (cfg.R + 2) * rhs
            else:
                x0 = torch.empty_like(rhs)
                S.electric_warm_start(ctx, net, x, rhs, x0)
            if x0 is not None:
                Lx = torch.empty_like(rhs)
                ctx.eval_electric(S.LAPLACE_DL, x0, Lx, S.OUT_COEF)
                r = rhs - (0.5 * x0 - (cfg.R - 1) / (cfg.R + 1) * Lx)
                r0[name].append(float(torch.linalg.norm(r) / torch.linalg.norm(rhs)))
            sol = torch.empty_like(rhs)
            it, res = ctx.gmres_solve(S.SYS_ELECTRIC, rhs, sol, x0=x0)
            assert res <= 1e-10
            counts[name].append(it)
            sols[name] = sol.cpu().numpy()
        for name in ("sphere", "learned"):
            assert np.abs(sols[name] - sols["zero"]).max() < 1e-8 * np.abs(sols["zero"]).max()
        ctx.close()
    mean = {k: float(np.mean(v)) for k, v in counts.items()}
    res0 = {k: float(np.mean(v)) for k, v in r0.items()}
    print("warm start: mean GMRES iterations", mean, "mean initial residual", res0)
    assert res0["learned"] < 0.5 * res0["sphere"], res0
    assert mean["learned"] <= mean["sphere"] < mean["zero"], mean
    net.close()
