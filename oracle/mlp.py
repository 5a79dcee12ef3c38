"""Multilayer perceptron for the learned GMRES warm start, plain numpy (test infrastructure only).

The paper has no learned component; this oracle defines the network the CUDA kernels
implement, so that their forward pass, gradients and optimiser step can be checked:
  h_0 = x;  h_l = tanh(bf16(h_{l-1}) bf16(W_l)^T + b_l) for hidden layers, the last layer
  linear;  loss = mean over the batch and outputs of (y - target)^2 / 2.
Weights are kept in FP32 ("master") and rounded to bfloat16 (round to nearest even) before
every product, as are the layer inputs; products accumulate in FP64 here (FP32 on the GPU).
Adam (Kingma & Ba) with bias correction updates the FP32 master weights.
"""
from __future__ import annotations

import numpy as np


def bf16(a):
    """Round float32 values to bfloat16 (nearest, ties to even) and return them as float32."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def forward(Ws, bs, x, rnd: bool = True):
    """Returns the list of layer outputs (h_0 = x, ..., h_L) and the (rounded) layer inputs.
    rnd=False skips the bfloat16 rounding and keeps FP64 throughout (used to pin the
    derivatives by finite differences)."""
    q = bf16 if rnd else (lambda a: np.asarray(a, dtype=np.float64))
    dt = np.float32 if rnd else np.float64
    hs = [np.asarray(x, dtype=dt)]
    ins = []
    L = len(Ws)
    for l in range(L):
        a = q(hs[-1]).astype(np.float64)
        ins.append(a)
        z = a @ q(Ws[l]).astype(np.float64).T + bs[l]
        hs.append((np.tanh(z) if l < L - 1 else z).astype(dt))
    return hs, ins


def loss_and_grads(Ws, bs, x, target, rnd: bool = True):
    """Loss = sum((y - t)^2) / (2 B) and its gradients w.r.t. the FP32 master weights and biases
    (straight-through: the bfloat16 rounding is treated as identity in the derivative)."""
    q = bf16 if rnd else (lambda a: np.asarray(a, dtype=np.float64))
    hs, ins = forward(Ws, bs, x, rnd)
    B = x.shape[0]
    y = hs[-1].astype(np.float64)
    d = (y - target) / B
    loss = 0.5 * float(((y - target) ** 2).sum()) / B
    gW = [None] * len(Ws)
    gb = [None] * len(Ws)
    L = len(Ws)
    for l in range(L - 1, -1, -1):
        if l < L - 1:
            d = d * (1.0 - hs[l + 1].astype(np.float64) ** 2)
        gW[l] = d.T @ ins[l]
        gb[l] = d.sum(axis=0)
        if l > 0:
            d = d @ q(Ws[l]).astype(np.float64)
    return loss, gW, gb


def adam(param, grad, m, v, t: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return param - lr * mh / (np.sqrt(vh) + eps), m, v


def init(widths, seed: int):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights from a seeded generator, zero biases."""
    rng = np.random.default_rng(seed)
    Ws, bs = [], []
    for a, b in zip(widths[:-1], widths[1:]):
        lim = 1.0 / np.sqrt(a)
        Ws.append(rng.uniform(-lim, lim, size=(b, a)).astype(np.float32))
        bs.append(np.zeros(b, dtype=np.float32))
    return Ws, bs
