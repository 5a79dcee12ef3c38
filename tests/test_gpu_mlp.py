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


@pytest.mark.parametrize("batch", [1, 3])
def test_few_row_inference_matches_oracle(S, batch):
    """Inference of 1-4 rows runs as matrix-vector products that read the weights once (odd K, so the rows
    of W start at every alignment); it computes the same function as the oracle's forward pass (inputs and
    weights rounded to bfloat16, FP32 sums): tolerance 1e-3 relative L2 against the FP64 sums of the same
    rounded values (an FP32 sum can flip the bfloat16 rounding of a hidden value, 2^-9 of it)."""
    widths = [8721, 96, 64, 131]
    Ws, bs = M.init(widths, 5)
    rng = np.random.default_rng(3)
    bs = [(b + 0.1 * rng.standard_normal(b.shape)).astype(np.float32) for b in bs]
    x = rng.standard_normal((batch, 8721)).astype(np.float32)
    net = S.MLP(widths, max_batch=8)
    for l in range(3):
        net.set_layer(l, Ws[l], bs[l])
    Y = torch.empty((batch, 131), device="cuda", dtype=torch.float32)
    net.forward(torch.tensor(x, device="cuda"), Y)
    hs, _ = M.forward(Ws, bs, x)
    assert rel(Y.cpu().numpy(), hs[-1]) < 1e-3
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
    """Train on solves of two-drop inputs made by the method itself (p = 6, 500 seeds; features from
    shbim_warm_start_features, targets the electric correction to the sphere solution and the Stokes
    velocity) and compare, on 12 held-out seeds: the electric initial residual of zero, sphere and
    sphere + network guesses (plain FP64 GMRES judges), and shbim_rates in mixed precision with and
    without the network as the context's warm start (inner iterations of both solves, same velocity)."""
    from paper_1811_10270_gb300 import warmstart
    p = 6
    Xtr, Ytr, its0 = warmstart.generate(inputs.config2(p=p, seed=sd, gap=0.1) for sd in range(1, 501))
    assert Xtr.shape[1] == 4 * 2 * 49 + 7 + 2 and Ytr.shape[1] == 4 * 2 * 49
    net, hist = warmstart.train(Xtr, Ytr, hidden=(256, 256, 256), epochs=150, batch=32, lr=1e-3)
    assert hist[-1] < 0.2 * hist[0]
    r0 = {"sphere": [], "learned": []}
    it_e = {"zero": [], "learned": []}
    rates_its = {"zero": [], "learned": []}
    for sd in range(100000, 100012):
        cfg = inputs.config2(p=p, seed=sd, gap=0.1)
        x = torch.tensor(np.concatenate([d.xcoef.ravel() for d in cfg.drops]), device="cuda")
        g = torch.tensor(np.concatenate([d.gamma_coef for d in cfg.drops]), device="cuda")
        nc = x.numel() // 3
        ph = warmstart.phys_of(cfg)
        ctx = S.Context(precision=S.FP64, R=cfg.R, gmres_tol=1e-10)
        ctx.set_drops([p, p], x, [d.lam for d in cfg.drops])
        rhs = torch.empty(nc, device="cuda", dtype=torch.float64)
        ctx.electric_rhs(cfg.E_u, rhs)
        feat = torch.empty(ctx.warm_start_feature_count(), device="cuda", dtype=torch.float32)
        ctx.warm_start_features(x, g, ph, feat)
        En0 = torch.empty_like(rhs)
        u0 = torch.empty(3 * nc, device="cuda", dtype=torch.float64)
        ctx.learned_guess(net, feat, rhs, En0, u0)
        sols = {}
        for name, x0 in (("zero", None), ("sphere", 3.0 * (cfg.R + 1) / (cfg.R + 2) * rhs), ("learned", En0)):
            if x0 is not None:
                Lx = torch.empty_like(rhs)
                ctx.eval_electric(S.LAPLACE_DL, x0, Lx, S.OUT_COEF)
                r = rhs - (0.5 * x0 - (cfg.R - 1) / (cfg.R + 1) * Lx)
                r0[name].append(float(torch.linalg.norm(r) / torch.linalg.norm(rhs)))
            sol = torch.empty_like(rhs)
            it, res = ctx.gmres_solve(S.SYS_ELECTRIC, rhs, sol, x0=x0)
            assert res <= 1e-10
            if name in it_e:
                it_e[name].append(it)
            sols[name] = sol.cpu().numpy()
        for name in ("sphere", "learned"):
            assert np.abs(sols[name] - sols["zero"]).max() < 1e-8 * np.abs(sols["zero"]).max()
        ctx.close()
        # the context's warm start inside shbim_rates (mixed precision)
        us = {}
        for name in ("zero", "learned"):
            ctx = S.Context(precision=S.FP32_COMP, R=cfg.R, gmres_tol=1e-10)
            ctx.set_drops([p, p], x, [d.lam for d in cfg.drops])
            ctx.set_warm_start(net if name == "learned" else None)
            u = torch.empty(3 * nc, device="cuda", dtype=torch.float64)
            gE = torch.empty(nc, device="cuda", dtype=torch.float64)
            rates_its[name].append(ctx.rates(ph, g, u, gE))
            us[name] = u.cpu().numpy()
            ctx.close()
        assert np.abs(us["learned"] - us["zero"]).max() < 1e-7 * np.abs(us["zero"]).max()
    res0 = {k: float(np.mean(v)) for k, v in r0.items()}
    it_mean = {k: np.mean(v, axis=0).tolist() for k, v in rates_its.items()}
    print("warm start: initial electric residual", res0, "FP64 electric iterations",
          {k: float(np.mean(v)) for k, v in it_e.items()}, "rates inner iterations [electric, Stokes]", it_mean)
    assert res0["learned"] < 0.5 * res0["sphere"], res0
    assert np.mean(it_e["learned"]) < np.mean(it_e["zero"])
    assert it_mean["learned"][1] < it_mean["zero"][1], it_mean      # the Stokes solve gains too
    net.close()
