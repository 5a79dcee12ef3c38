"""Restarted GMRES in FP64 (test infrastructure only).

The paper solves its Galerkin systems without naming the solver; this is the textbook
restarted GMRES(m) (Saad & Schultz) with modified Gram-Schmidt Arnoldi and Givens rotations,
stopping when the true relative residual ||b - A x|| / ||b|| reaches tol.
"""
from __future__ import annotations

import numpy as np


def gmres(matvec, b, x0=None, tol: float = 1e-8, restart: int = 50, maxiter: int = 500):
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n), {"iters": 0, "resid": 0.0, "history": [0.0]}
    hist = []
    total = 0
    while total < maxiter:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta / bnorm <= tol:
            break
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        k_used = 0
        for k in range(restart):
            w = matvec(V[k])
            for i in range(k + 1):
                H[i, k] = np.dot(w, V[i])
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] != 0.0:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):
                a, c = H[i, k], H[i + 1, k]
                H[i, k] = cs[i] * a + sn[i] * c
                H[i + 1, k] = -sn[i] * a + cs[i] * c
            den = np.hypot(H[k, k], H[k + 1, k])
            cs[k] = H[k, k] / den
            sn[k] = H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            total += 1
            k_used = k + 1
            hist.append(abs(g[k + 1]) / bnorm)
            if abs(g[k + 1]) / bnorm <= tol or total >= maxiter:
                break
        y = np.linalg.solve(np.triu(H[:k_used, :k_used]), g[:k_used])
        x = x + V[:k_used].T @ y
    r = b - matvec(x)
    return x, {"iters": total, "resid": float(np.linalg.norm(r) / bnorm), "history": hist}
