"""Seeded synthetic drop configurations shared by the oracle, the tests and the bench.

This module is data only: it draws random numbers and lays them out in the coefficient
layout that both the oracle and the CUDA library document (real orthonormal spherical
harmonics, index n*n + n + m, Condon-Shortley phase). It performs none of the method's
arithmetic: no transforms, no quadrature, no surface evaluation.

Real basis (used by every consumer):
    S_n0  = Pbar_n^0(cos t)
    S_nm  = sqrt(2) Pbar_n^m(cos t) cos(m f)      (m > 0)
    S_n-m = sqrt(2) Pbar_n^m(cos t) sin(m f)      (m > 0)
with Pbar_n^m = sqrt((2n+1)/(4 pi) (n-m)!/(n+m)!) P_n^m and P_n^m carrying (-1)^m
(the normalised harmonics and Legendre functions of Section 2 of the paper).

In that basis the unit sphere x = (sin t cos f, sin t sin f, cos t) has the coefficients
x: -sqrt(4 pi/3) on S_11, y: -sqrt(4 pi/3) on S_1-1, z: +sqrt(4 pi/3) on S_10, and a
constant c has sqrt(4 pi) c on S_00.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SQRT_4PI = math.sqrt(4.0 * math.pi)
SQRT_4PI_3 = math.sqrt(4.0 * math.pi / 3.0)


def ncoef(p: int) -> int:
    """Number of real coefficients of a degree-p expansion."""
    return (p + 1) * (p + 1)


def idx(n: int, m: int) -> int:
    return n * n + n + m


@dataclass
class Drop:
    p: int
    xcoef: np.ndarray          # (3, (p+1)^2) float64, absolute positions
    gamma_coef: np.ndarray     # ((p+1)^2,) surfactant concentration
    lam: float                 # viscosity ratio of this drop
    centre: np.ndarray         # (3,) the centre used to place it (= xcoef[:,0]/sqrt(4 pi))
    radius: float


@dataclass
class Config:
    name: str
    drops: list
    R: float                   # conductivity ratio
    Q: float                   # permittivity ratio
    E_u: np.ndarray            # uniform field vector
    E_quad: float = 0.0        # quadrupole strength (E = E_quad*(x, -y, 0)) when used
    Ca_E: float = 0.1
    meta: dict = field(default_factory=dict)


def sphere_coef(p: int, radius: float = 1.0, centre=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Coefficients of a sphere of the given radius and centre, degree-p layout."""
    c = np.zeros((3, ncoef(p)))
    c[0, idx(1, 1)] = -SQRT_4PI_3 * radius
    c[1, idx(1, -1)] = -SQRT_4PI_3 * radius
    c[2, idx(1, 0)] = SQRT_4PI_3 * radius
    for k in range(3):
        c[k, 0] = SQRT_4PI * centre[k]
    return c


def perturbed_coef(p: int, rng: np.random.Generator, radius: float, centre,
                   amp: float = 0.05, lmax: int = 8) -> np.ndarray:
    """Sphere plus a random smooth perturbation of every position component:
    coefficient (n, m) of each component ~ N(0,1) * amp / n^2 * radius, 1 <= n <= lmax."""
    c = sphere_coef(p, radius, centre)
    for n in range(1, min(lmax, p) + 1):
        for m in range(-n, n + 1):
            c[:, idx(n, m)] += rng.standard_normal(3) * amp / (n * n) * radius
    return c


def gamma_random(p: int, rng: np.random.Generator, amp: float = 0.2, lmax: int = 4) -> np.ndarray:
    """Surfactant 1 + perturbation on 1 <= n <= lmax; each coefficient ~ U(-amp, amp)/24."""
    g = np.zeros(ncoef(p))
    g[0] = SQRT_4PI
    for n in range(1, min(lmax, p) + 1):
        for m in range(-n, n + 1):
            g[idx(n, m)] = rng.uniform(-amp, amp) / 24.0
    return g


def config1(p: int = 16) -> Config:
    """Single unit sphere, lambda=1, R=0.1, Q=1, E=(0,0,1), Gamma = 1 + 0.1 Y_2^0."""
    g = np.zeros(ncoef(p))
    g[0] = SQRT_4PI
    if p >= 2:
        g[idx(2, 0)] = 0.1
    d = Drop(p=p, xcoef=sphere_coef(p), gamma_coef=g, lam=1.0,
             centre=np.zeros(3), radius=1.0)
    return Config("single unit sphere p=%d" % p, [d], R=0.1, Q=1.0,
                  E_u=np.array([0.0, 0.0, 1.0]))


def config2(p: int = 32, seed: int = 0, gap: float = 0.1) -> Config:
    """Two perturbed unit drops, centres (0,0,+-(1+gap/2)), lambda=5, R=2, Q=0.5."""
    rng = np.random.default_rng(seed)
    drops = []
    h = 1.0 + 0.5 * gap
    for s in (-1.0, 1.0):
        ctr = np.array([0.0, 0.0, s * h])
        drops.append(Drop(p=p, xcoef=perturbed_coef(p, rng, 1.0, ctr),
                          gamma_coef=gamma_random(p, rng), lam=5.0,
                          centre=ctr, radius=1.0))
    return Config("two drops p=%d gap=%g seed=%d" % (p, gap, seed), drops, R=2.0, Q=0.5,
                  E_u=np.array([0.0, 0.0, 1.0]), meta={"seed": seed})


def _place(rng: np.random.Generator, radii, box: float, gap: float):
    """Centres uniform in the box (each sphere inside it), rejection-sampled so that nominal
    spheres are at least `gap` apart."""
    centres = []
    for i in range(len(radii)):
        for _ in range(100000):
            c = rng.uniform(-box / 2 + radii[i], box / 2 - radii[i], size=3)
            if all(np.linalg.norm(c - centres[j]) >= radii[i] + radii[j] + gap for j in range(len(centres))):
                centres.append(c)
                break
        else:
            raise RuntimeError("could not place drop %d" % i)
    return centres


def config3(seed: int = 3, n_drops: int = 64, box: float = 12.0, min_gap: float = 0.2,
            degrees=(16, 24, 32, 48), slack: float = 0.2) -> Config:
    """Many drops of uneven degree in a cubic box; centres by rejection sampling so that the
    nominal spheres are at least min_gap + slack apart (slack covers the perturbation)."""
    rng = np.random.default_rng(seed)
    ps = rng.choice(np.array(degrees), size=n_drops)
    radii = rng.uniform(0.8, 1.2, size=n_drops)
    centres = _place(rng, radii, box, min_gap + slack)
    drops = []
    for i in range(n_drops):
        p = int(ps[i])
        drops.append(Drop(p=p, xcoef=perturbed_coef(p, rng, float(radii[i]), centres[i]),
                          gamma_coef=gamma_random(p, rng), lam=float(rng.uniform(0.5, 10.0)),
                          centre=np.asarray(centres[i]), radius=float(radii[i])))
    return Config("batched %d drops p in %s seed=%d" % (n_drops, list(degrees), seed), drops,
                  R=2.0, Q=0.5, E_u=np.array([0.0, 0.0, 1.0]), meta={"seed": seed})


def config5(seed: int = 5, n_drops: int = 16, p: int = 64, box: float = 8.0, min_gap: float = 0.2,
            slack: float = 0.2) -> Config:
    """16 unit drops of degree 64 (perturbed as above) in an 8^3 box, nominal gaps >= min_gap +
    slack, lambda = 1, R = 4.5, Q = 5, quadrupole field E = (x, -y, 0), surfactant as above
    (the Peclet number 10 is a time-step parameter, not part of the inputs)."""
    rng = np.random.default_rng(seed)
    radii = np.ones(n_drops)
    centres = _place(rng, radii, box, min_gap + slack)
    drops = [Drop(p=p, xcoef=perturbed_coef(p, rng, 1.0, centres[i]), gamma_coef=gamma_random(p, rng),
                  lam=1.0, centre=np.asarray(centres[i]), radius=1.0) for i in range(n_drops)]
    return Config("%d drops p=%d quadrupole field seed=%d" % (n_drops, p, seed), drops, R=4.5, Q=5.0,
                  E_u=np.array([0.0, 0.0, 0.0]), E_quad=1.0, meta={"seed": seed})


def random_density(p: int, rng: np.random.Generator, ncomp: int = 1, decay: float = 1.0) -> np.ndarray:
    """Random smooth density coefficients (ncomp, (p+1)^2): N(0,1)/(n+1)^decay."""
    out = np.zeros((ncomp, ncoef(p)))
    for n in range(p + 1):
        for m in range(-n, n + 1):
            out[:, idx(n, m)] = rng.standard_normal(ncomp) / (n + 1.0) ** decay
    return out
