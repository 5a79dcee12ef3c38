"""Training driver of the learned warm start (host orchestration only; every feature, product,
activation, gradient and optimiser step runs in libshbim's kernels).

Samples are drop configurations the caller supplies (objects with `drops`, each drop having `p`,
`xcoef`, `gamma_coef` and `lam`, plus `R`, `Q`, `Ca_E`, `E_u` and `E_quad`), all of one layout. Each is
solved by the library itself to a tight tolerance, so the network learns from the method: the features
are the library's warm-start features (positions, surfactant, field, lambda, R, Q, Ca_E); the targets are
the electric solution's correction to the sphere solution 3(R+1)/(R+2) rhs and the velocity of the
Stokes solve (shbim_rates), 4 ncoef values. Inputs and targets are standardised for training and the
standardisation is attached to the network afterwards -- the input part as the network's FP32 input
affine (applied before the first bfloat16 rounding: raw coefficients near 2 would lose the
0.05-sized perturbations to bfloat16), the output part folded into the last layer -- so the deployed
network maps raw features to raw guesses (shbim_learned_guess).
"""
from __future__ import annotations

import math

import numpy as np

from . import FP32_COMP, SYS_ELECTRIC, Context, MLP, phys


def phys_of(cfg, inner_tol: float = 1e-5):
    """The physical parameters of a configuration (Langmuir beta 0.2, x_s 0.5)."""
    return phys(R=cfg.R, Q=cfg.Q, Ca_E=cfg.Ca_E, beta=0.2, x_s=0.5, E_u=tuple(cfg.E_u), E_q=cfg.E_quad,
                inner_tol=inner_tol, Pe=math.inf)


def generate(configs, tol: float = 1e-10):
    """(features [n, F], targets [n, 4 ncoef], inner iterations from zero [n, 2]) for the given drop
    configurations (all of one layout): mixed-precision solves refined to `tol`."""
    import torch
    dev = torch.device("cuda")
    X, Y, its = [], [], []
    ctx = None
    for cfg in configs:
        if ctx is None:
            ctx = Context(precision=FP32_COMP, R=cfg.R, gmres_tol=tol)
        x = torch.tensor(np.concatenate([d.xcoef.ravel() for d in cfg.drops]), device=dev)
        g = torch.tensor(np.concatenate([d.gamma_coef for d in cfg.drops]), device=dev)
        ctx.set_drops([d.p for d in cfg.drops], x, [d.lam for d in cfg.drops])
        nc = x.numel() // 3
        ph = phys_of(cfg)
        feat = torch.empty(ctx.warm_start_feature_count(), device=dev, dtype=torch.float32)
        ctx.warm_start_features(x, g, ph, feat)
        rhs = torch.empty(nc, device=dev, dtype=torch.float64)
        ctx.set_R(cfg.R)
        ctx.electric_rhs(cfg.E_u, rhs, E_q=cfg.E_quad)
        En = torch.empty_like(rhs)
        ctx.gmres_solve_refined(SYS_ELECTRIC, rhs, En)
        u = torch.empty(3 * nc, device=dev, dtype=torch.float64)
        gE = torch.empty(nc, device=dev, dtype=torch.float64)
        it = ctx.rates(ph, g, u, gE)
        c = 3.0 * (cfg.R + 1.0) / (cfg.R + 2.0)
        X.append(feat.cpu().numpy())
        Y.append(torch.cat([En - c * rhs, u]).cpu().numpy().astype(np.float32))
        its.append(it)
    ctx.close()
    return np.stack(X), np.stack(Y), np.array(its)


def init_layers(widths, rng: np.random.Generator):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases (seeded data)."""
    out = []
    for a, b in zip(widths[:-1], widths[1:]):
        lim = 1.0 / np.sqrt(a)
        out.append((rng.uniform(-lim, lim, size=(b, a)).astype(np.float32), np.zeros(b, np.float32)))
    return out


def train(X, Y, hidden=(512, 512, 512), epochs: int = 200, batch: int = 64, lr: float = 1e-3, seed: int = 0):
    """Train on (X, Y); returns (net, history of epoch losses). The returned network takes raw
    features and produces raw targets. Targets are standardised per output (the electric and velocity
    blocks have different sizes)."""
    import torch
    dev = torch.device("cuda")
    mu, sd = X.mean(0), X.std(0)
    sd = np.where(sd > 1e-6, sd, 1.0).astype(np.float32)
    ym = Y.mean(0)
    ys = Y.std(0)
    ys = np.where(ys > 1e-3 * (ys.max() + 1e-30), ys, 1e-3 * (ys.max() + 1e-30)).astype(np.float32)
    Xn = torch.tensor((X - mu) / sd, device=dev)
    Yn = torch.tensor((Y - ym) / ys, device=dev)
    widths = [X.shape[1], *hidden, Y.shape[1]]
    net = MLP(widths, max_batch=max(batch, 1))
    rng = np.random.default_rng(seed)
    for l, (W, b) in enumerate(init_layers(widths, rng)):
        net.set_layer(l, W, b)
    n = X.shape[0]
    hist = []
    for ep in range(epochs):
        perm = torch.tensor(rng.permutation(n), device=dev)
        tot = 0.0
        for i in range(0, n - batch + 1, batch):
            idx = perm[i:i + batch]
            tot += net.train_step(Xn[idx].contiguous(), Yn[idx].contiguous(), lr)
        hist.append(tot / max(1, n // batch))
    # attach the standardisation: input affine in FP32, output scaling folded into the last layer
    L = len(widths) - 1
    net.set_input_affine(mu.astype(np.float32), (1.0 / sd).astype(np.float32))
    WL, bL, _, _ = net.get_layer(L - 1)
    net.set_layer(L - 1, WL * ys[:, None], bL * ys + ym)
    return net, hist
