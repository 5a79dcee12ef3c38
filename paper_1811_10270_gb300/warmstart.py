"""Training driver of the learned electric warm start (host orchestration only; every
product, activation, gradient and optimiser step runs in libshbim's kernels).

Samples are drop configurations the caller supplies (objects with `drops`, each drop having `p`,
`xcoef` and `lam`, plus the conductivity ratio `R` and the uniform field `E_u`); each is solved by
the library's own FP64 GMRES, so the network learns from the method itself.
Inputs are the position coefficients of both drops; targets are the correction of E_n to the
sphere solution 3(R+1)/(R+2) rhs. Inputs and targets are standardised for training and the
standardisation is then attached to the network -- the input part as the network's FP32
input affine (applied before the first bfloat16 rounding: raw coefficients near 2 would lose
the 0.05-sized perturbations to bfloat16), the output part folded into the last layer -- so
that the deployed network maps raw coefficients to the raw correction.
"""
from __future__ import annotations

import numpy as np

from . import FP64, SYS_ELECTRIC, Context, MLP


def generate(configs, tol: float = 1e-10):
    """(features [n, 3 ncoef], targets [n, ncoef], iterations from zero) for the given drop
    configurations (all of one layout)."""
    import torch
    dev = torch.device("cuda")
    X, Y, its = [], [], []
    ctx = None
    for cfg in configs:
        if ctx is None:
            ctx = Context(precision=FP64, R=cfg.R, gmres_tol=tol)
        x = np.concatenate([d.xcoef.ravel() for d in cfg.drops])
        xd = torch.tensor(x, device=dev)
        ctx.set_drops([d.p for d in cfg.drops], xd, [d.lam for d in cfg.drops])
        nc = xd.numel() // 3
        rhs = torch.empty(nc, device=dev, dtype=torch.float64)
        ctx.electric_rhs(cfg.E_u, rhs)
        sol = torch.empty_like(rhs)
        it, _ = ctx.gmres_solve(SYS_ELECTRIC, rhs, sol)
        c = 3.0 * (cfg.R + 1.0) / (cfg.R + 2.0)
        X.append(x.astype(np.float32))
        Y.append((sol - c * rhs).cpu().numpy().astype(np.float32))
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
    inputs and produces raw targets."""
    import torch
    dev = torch.device("cuda")
    mu, sd = X.mean(0), X.std(0)
    sd = np.where(sd > 1e-6, sd, 1.0).astype(np.float32)
    ym, ys = Y.mean(0), float(Y.std()) + 1e-12
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
    net.set_layer(L - 1, WL * ys, bL * ys + ym)
    return net, hist
