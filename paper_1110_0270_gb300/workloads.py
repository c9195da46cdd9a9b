"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds no lattice Boltzmann arithmetic: it only draws numbers and
describes the paper's set-ups (sizes, Reynolds numbers, initial density and
velocity fields).  Both the CUDA path and the FP64 oracle receive the arrays
it returns; each converts viscosity to its relaxation coefficient itself.

Set-ups (Sections 6-8 of the paper, sizes as in the benchmark configurations):
  * shock tube: D1Q3, 800 sites, rho = 1 on the left half and 0.5 on the
    right, u = 0;
  * shear wave: D2Q9 periodic L x L, rho = 1, u_x = 0, u_y = u0 sin(2 pi x / L);
  * lid-driven cavity: D2Q9 N x N, rho = 1, u = 0, top wall moving with U,
    nu = U (N - 1) / Re;
  * batched cavities: side lengths uniform in [64, 768], Re log-uniform in
    [100, 20000], drawn from numpy's default_rng(seed).
"""
from __future__ import annotations

import numpy as np


def shock_tube(n: int = 800, nu: float = 1e-9) -> tuple[dict, dict]:
    """D1Q3 shock tube of Section 6: density 1 on sites 1..n/2, 0.5 after."""
    rho = np.where(np.arange(n) < n // 2, 1.0, 0.5)[None, :]
    cfg = dict(lattice="D1Q3", nx=n, ny=1, bc="ends", nu=nu, lid_u=0.0)
    return cfg, dict(rho=rho, ux=np.zeros_like(rho), uy=np.zeros_like(rho))


def shear_wave(L: int = 64, u0: float = 0.05, nu: float = 0.01) -> tuple[dict, dict]:
    """Periodic shear wave of Section 7 on an L x L grid (x = 0..L-1)."""
    x = np.arange(L, dtype=np.float64)
    uy = np.tile(u0 * np.sin(2.0 * np.pi * x / L), (L, 1))
    rho = np.ones((L, L))
    cfg = dict(lattice="D2Q9", nx=L, ny=L, bc="periodic", nu=nu, lid_u=0.0)
    return cfg, dict(rho=rho, ux=np.zeros_like(rho), uy=uy)


def shear_decay(L: int, re: float, u0: float = 0.05, points: int | None = None) -> tuple[dict, dict]:
    """Section 7's shear-decay set-up: a periodic square of `points` (L + 1 by
    default, the paper's count) sites a side, rho = 1, u_x = 0,
    u_y = u0 sin(2 pi x / L), viscosity from Re = u0 L / nu."""
    n = L + 1 if points is None else points
    x = np.arange(n, dtype=np.float64)
    uy = np.tile(u0 * np.sin(2.0 * np.pi * x / L), (n, 1))
    rho = np.ones((n, n))
    cfg = dict(lattice="D2Q9", nx=n, ny=n, bc="periodic", nu=u0 * L / re, lid_u=0.0)
    return cfg, dict(rho=rho, ux=np.zeros_like(rho), uy=uy)


def cavity(n: int, re: float, lid_u: float) -> tuple[dict, dict]:
    """Lid-driven cavity of Section 8: fluid at rest, lid speed lid_u,
    viscosity from Re = lid_u (n - 1) / nu."""
    rho = np.ones((n, n))
    cfg = dict(lattice="D2Q9", nx=n, ny=n, bc="cavity", nu=lid_u * (n - 1) / re, lid_u=lid_u)
    return cfg, dict(rho=rho, ux=np.zeros_like(rho), uy=np.zeros_like(rho))


def random_fields(ny: int, nx: int, seed: int, rho_amp: float = 0.05,
                  u_amp: float = 0.05) -> dict:
    """Smooth-free random density and velocity fields (uniform noise)."""
    rng = np.random.default_rng(seed)
    return dict(rho=1.0 + rho_amp * rng.uniform(-1, 1, (ny, nx)),
                ux=u_amp * rng.uniform(-1, 1, (ny, nx)),
                uy=u_amp * rng.uniform(-1, 1, (ny, nx)))


def lognormal_factors(shape: tuple, seed: int, amp: float) -> np.ndarray:
    """exp(amp * N(0, 1)) factors; multiplied into a state by the caller to
    put sites out of equilibrium with positive populations."""
    rng = np.random.default_rng(seed)
    return np.exp(amp * rng.standard_normal(shape))


def normal_noise(shape: tuple, seed: int, sigma: float) -> np.ndarray:
    """sigma * N(0, 1) samples (additive perturbation of a state)."""
    return sigma * np.random.default_rng(seed).standard_normal(shape)


def hot_spots(ny: int, nx: int, seed: int, count: int, amp: float) -> np.ndarray:
    """Per-site amplitude field that is zero except at `count` random sites,
    where it is amp * U(0.5, 1): used to plant a few strongly
    non-equilibrium sites (limiter candidates) in an otherwise smooth state."""
    rng = np.random.default_rng(seed)
    a = np.zeros(ny * nx)
    idx = rng.choice(ny * nx, size=min(count, ny * nx), replace=False)
    a[idx] = amp * rng.uniform(0.5, 1.0, idx.size)
    return a.reshape(ny, nx)


def batched_cavities(n: int = 512, seed: int = 0, side_lo: int = 64, side_hi: int = 768,
                     re_lo: float = 100.0, re_hi: float = 20000.0) -> list[dict]:
    """Instance list of the batched configuration."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(side_lo, side_hi + 1, size=n)
    res = np.exp(rng.uniform(np.log(re_lo), np.log(re_hi), size=n))
    kinds = ["lbgk", "elbm", "ehrenfest", "median"]
    return [dict(side=int(s), re=float(r), collision=kinds[j % 4]) for j, (s, r) in
            enumerate(zip(sides, res))]
