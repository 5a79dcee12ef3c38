"""Band-limited fields on the rotated grids of all targets, fast form; plain FP64 numpy (test
infrastructure only).

Section 2.1: the singular rule needs, for every target x0 = x(theta0, phi0), the density and the geometry
on the grid rotated so that the target is its north pole, R = Rz(phi0) Ry(theta0). The paper notes a fast
algorithm for these rotations over all targets (Gimbutas and Veerapaneni, O(p^4 log p) for the O(p^2)
targets of a drop); this module is an algorithm of that cost written from the structure of the problem:

  * targets of one latitude theta0 differ only in phi0 = 2 pi l / L (the L = 2p+2 grid longitudes): the
    rotated node R x_jk has the polar angle theta' of y = Ry(theta0) x_jk and the longitude phi' + phi0;
  * with f(theta, phi) = sum_m C_m(theta) e^{i m phi}, the values for all targets of the latitude are
        f(R_l x_jk) = sum_m [C_m(theta'_jk) e^{i m phi'_jk}] e^{i m phi0_l},
    one DFT over m per rotated node (m folded modulo L, then an FFT over the L targets);
  * C_m(theta) = sum_n a_nm Pbar_n^m(cos theta) is a trigonometric polynomial of degree p in theta when
    sin theta keeps its sign on (pi, 2 pi) (Pbar_n^m carries sin^m theta), so its Fourier coefficients
    come from an FFT of samples on the whole circle, and its values at the O(p^2) angles theta' of a
    latitude from a type-2 non-uniform FFT (Gaussian gridding after Dutt and Rokhlin, in the form of
    Greengard and Lee: deconvolve, one FFT onto an oversampled grid, Gaussian interpolation).
Per latitude O(p^3 (w + log p)) with w the interpolation width, for the p + 1 latitudes O(p^4 (w + log p))
against the O(p^5) of one rotation per target. `self_values` applies it to the singular rule of
oracle.quadrature (Eq. mod_weights) for every target of a drop.
"""
from __future__ import annotations

import math

import numpy as np

from . import quadrature, sh

MSP = 16          # Gaussian interpolation half-width, in fine-grid points (~1e-15 relative)
OVERSAMPLE = 2    # fine grid / number of modes


def theta_fourier(coef, p: int) -> tuple[np.ndarray, np.ndarray]:
    """Fourier coefficients in theta of C_m(theta), m = -p..p, for the real degree-p expansion coef.
    Returns (B, ms): B[i, s] for m = ms[i] and frequency s in np.fft order over T = 2p + 2 samples."""
    T = 2 * p + 2
    th = 2.0 * math.pi * np.arange(T) / T
    P = sh.alf(p, np.cos(th), np.sin(th))            # signed sin theta: the trigonometric continuation
    coef = np.asarray(coef, dtype=np.float64)
    ms = np.arange(-p, p + 1)
    C = np.zeros((ms.size, T), dtype=np.complex128)
    for n in range(p + 1):
        C[p] += coef[sh.idx(n, 0)] * P[n, 0]
        for m in range(1, n + 1):
            # real basis: sqrt2 Pbar (a_nm cos m phi + a_n,-m sin m phi) = C_m e^{i m phi} + C_-m e^{-i m phi}
            half = (sh.SQRT2 / 2.0) * P[n, m]
            C[p + m] += half * (coef[sh.idx(n, m)] - 1j * coef[sh.idx(n, -m)])
            C[p - m] += half * (coef[sh.idx(n, m)] + 1j * coef[sh.idx(n, -m)])
    return np.fft.fft(C, axis=1) / T, ms


def nufft2(B: np.ndarray, x: np.ndarray, msp: int = MSP, R: int = OVERSAMPLE) -> np.ndarray:
    """sum_s B[:, s] e^{i s x_j} at the angles x (rows of B in np.fft frequency order): deconvolve by
    the Gaussian's Fourier coefficients, synthesise on a grid R times finer, and interpolate with the
    periodic Gaussian g(d) = exp(-d^2 / (4 tau)), tau = pi msp / (M^2 R (R - 1/2))."""
    M = B.shape[1]
    Mr = R * M
    tau = math.pi * msp / (M * M * R * (R - 0.5))
    s = np.fft.fftfreq(M, 1.0 / M)
    Bt = B * (math.sqrt(math.pi / tau) * np.exp(s * s * tau))
    fine = np.zeros((B.shape[0], Mr), dtype=np.complex128)
    fine[:, (s.astype(int)) % Mr] = Bt
    vals = np.fft.ifft(fine, axis=1) * Mr           # f_{-tau} on y_m = 2 pi m / Mr
    h = 2.0 * math.pi / Mr
    x = np.asarray(x, dtype=np.float64) % (2.0 * math.pi)
    m0 = np.floor(x / h).astype(int)
    offs = np.arange(-msp + 1, msp + 1)
    idx = m0[:, None] + offs[None, :]                # (K, 2 msp)
    d = x[:, None] - idx * h
    g = np.exp(-d * d / (4.0 * tau)) / Mr
    return np.einsum("ikw,kw->ik", vals[:, idx % Mr], g)


def rotated_values(coef, p: int, q: int, theta0: float, L: int, msp: int = MSP) -> np.ndarray:
    """Values of the degree-p expansion coef on the degree-q grid rotated by Rz(2 pi l / L) Ry(theta0),
    l = 0..L-1: array (L, (q+1)(2q+2)) in the grid's [j][k] order."""
    B, ms = theta_fourier(coef, p)
    y = quadrature.rotation(theta0, 0.0) @ quadrature.unit_grid(q)
    thp = np.arccos(np.clip(y[2], -1.0, 1.0))
    php = np.arctan2(y[1], y[0])
    G = nufft2(B, thp, msp) * np.exp(1j * ms[:, None] * php[None, :])      # (2p+1, Nq)
    folded = np.zeros((L, G.shape[1]), dtype=np.complex128)
    np.add.at(folded, ms % L, G)
    return (np.fft.ifft(folded, axis=0) * L).real


def self_values(xcoef, p: int, dens, kind: str, q: int | None = None) -> np.ndarray:
    """The singular rule of oracle.quadrature.self_rows (kind 'lsl', 'ladl', 'sto_s' or 'sto_d') applied to
    the density coefficients dens ((ncoef,) or (3, ncoef)) at every target of the degree-p grid, with all
    rotated values from rotated_values: the density and x (degree p), and J n (the area element times
    the normal, a function on the parameter sphere independent of how it is rotated, of degree at most
    2p + 1, expanded exactly on the degree 2p + 1 grid). Returns (ntargets,) or (3, ntargets)."""
    from . import geometry
    q = 2 * p + 1 if q is None else q
    xcoef = np.asarray(xcoef, dtype=np.float64).reshape(3, -1)
    dens = np.asarray(dens, dtype=np.float64)
    Q = 2 * p + 1
    _, nQ, JQ = geometry.surface_on_grid(xcoef, p, Q)
    jn = sh.sht_forward(JQ * nQ, Q, Q)                       # (3, (Q+1)^2)
    x0s, n0s, _ = geometry.surface_on_grid(xcoef, p, p)
    L = 2 * p + 2
    mu = quadrature.modified_weights(q) * quadrature.INV4PI
    _, _, thetas, _ = sh.gauss_grid(p)
    vector = dens.ndim == 2
    out = np.zeros((3, x0s.shape[1]) if vector else x0s.shape[1])
    for i, th0 in enumerate(thetas):
        X = np.stack([rotated_values(xcoef[c], p, q, th0, L) for c in range(3)])      # (3, L, Nq)
        JN = np.stack([rotated_values(jn[c], Q, q, th0, L) for c in range(3)])
        D = np.stack([rotated_values(dens[c], p, q, th0, L) for c in range(3)]) if vector \
            else rotated_values(dens, p, q, th0, L)
        J = np.sqrt((JN * JN).sum(axis=0))
        for l in range(L):
            t = i * L + l
            x0, n0 = x0s[:, t], n0s[:, t]
            w = mu * J[l]
            if vector:
                K = quadrature.kernel_tensor(kind, x0, X[:, l], JN[:, l] / J[l])
                out[:, t] = np.einsum("iks,ks->i", K, D[:, l] * w)
            else:
                out[t] = (quadrature.kernel_scalar(kind, x0, n0, X[:, l]) * D[l] * w).sum()
    return out
