"""Seeded synthetic input fields for the PonD step.

This module holds no arithmetic of the method itself: it only draws the
macroscopic fields (density, velocity, temperature) that both the CUDA path
and the CPU oracle start from.  Each side builds its own populations from
these fields.  All draws use NumPy's PCG64 with the base seed 1806050890
plus the workload number.

Workloads (shapes follow the paper's incompressible Taylor-Green vortex,
App. D, and its compressible advected flows):

1. ``tg64``          64 x 64 Taylor-Green, rho = 1, T = 1, u0 = 0.05, nu = 0.01
2. ``supersonic``    N x N (2048 at scale), uniform u = (1.5, 0.5), rho and T
                     = 1 + a sum of 8 seeded sinusoids (0.1/8 each, integer
                     wavenumbers 1..8)
3. ``precision``     N x N (4096 at scale), same u, T = 2^s with s a
                     normalised sum of 8 seeded sinusoids (T in [0.5, 2]) at
                     constant pressure: rho = (1 + the 8-mode perturbation) / T
4. ``adjoint``       512 x 512 Taylor-Green u0 = 0.3 plus a Gaussian density
                     pulse (amplitude 0.2, sigma 16), and a seeded target
6. ``vortex``        isentropic vortex u_phi = Ma_v c r exp((1 - r^2)/2), r = r'/R,
                     c = sqrt(2 T_inf), advected by U = Ma_a c (main text,
                     vortex benchmark); T and rho from radial equilibrium of
                     an isentropic gamma = 2 gas
5. ``ensemble``      256 grids with sides in 32..512, Mach 0..3 in a random
                     direction, T ratio r in [0.5, 4]: T = 1 + (r-1) s(x),
                     s in [0, 1] from 8 modes of wavenumber <= 2 per side (so
                     a 32-cell grid still resolves the ratio-4 variation)
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BASE_SEED = 1806050890


def rng(workload: int, sub: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([BASE_SEED + workload, sub]))


@dataclass
class Fields:
    rho: np.ndarray  # (ny, nx) float64
    ux: np.ndarray
    uy: np.ndarray
    T: np.ndarray

    @property
    def shape(self):
        return self.rho.shape


def _grid(nx: int, ny: int):
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    return np.meshgrid(x, y)  # X[y, x], Y[y, x]


def sinusoids(nx: int, ny: int, g: np.random.Generator, modes: int = 8,
              kmax: int = 8) -> np.ndarray:
    """Sum of ``modes`` unit-amplitude sinusoids sin(2 pi (kx x/nx + ky y/ny) + phi)
    with integer wavenumber components in [-kmax, kmax], max(|kx|,|ky|) >= 1,
    and uniform random phases."""
    X, Y = _grid(nx, ny)
    out = np.zeros((ny, nx))
    for _ in range(modes):
        while True:
            kx, ky = g.integers(-kmax, kmax + 1, size=2)
            if max(abs(kx), abs(ky)) >= 1:
                break
        phi = g.uniform(0.0, 2.0 * np.pi)
        out += np.sin(2.0 * np.pi * (kx * X / nx + ky * Y / ny) + phi)
    return out


def taylor_green(nx: int, ny: int, u0: float, rho: float = 1.0, T: float = 1.0) -> Fields:
    """u_x = -(u0/sqrt 2) cos(kx) sin(ky), u_y = (u0/sqrt 2) sin(kx) cos(ky),
    k = 2 pi / L (App. D; square grids use one k, otherwise k per axis)."""
    X, Y = _grid(nx, ny)
    kx = 2.0 * np.pi / nx
    ky = 2.0 * np.pi / ny
    a = u0 / np.sqrt(2.0)
    ux = -a * np.cos(kx * X) * np.sin(ky * Y)
    uy = a * np.sin(kx * X) * np.cos(ky * Y)
    return Fields(np.full((ny, nx), rho), ux, uy, np.full((ny, nx), T))


def tg64(n: int = 64) -> Fields:
    return taylor_green(n, n, 0.05)


def supersonic(n: int = 2048, nx: int | None = None, ny: int | None = None) -> Fields:
    nx = nx or n
    ny = ny or n
    g = rng(2)
    rho = 1.0 + (0.1 / 8.0) * sinusoids(nx, ny, g)
    T = 1.0 + (0.1 / 8.0) * sinusoids(nx, ny, g)
    return Fields(rho, np.full((ny, nx), 1.5), np.full((ny, nx), 0.5), T)


def precision(n: int = 4096) -> Fields:
    """T = 2^s (ratio 4 across the field) at constant pressure: rho = (1 +
    the 8-mode perturbation) / T, so the temperature variation is an advected
    entropy mode rather than a pressure jump that would steepen into shocks."""
    g = rng(3)
    pert = 1.0 + (0.1 / 8.0) * sinusoids(n, n, g)
    s = sinusoids(n, n, g)
    s /= np.abs(s).max()
    T = np.exp2(s)
    return Fields(pert / T, np.full((n, n), 1.5), np.full((n, n), 0.5), T)


def adjoint(n: int = 512):
    """Initial fields and target density of the adjoint workload."""
    f = taylor_green(n, n, 0.3)
    X, Y = _grid(n, n)
    c = n / 2.0
    dx = X - c
    dy = Y - c
    pulse = 0.2 * np.exp(-(dx * dx + dy * dy) / (2.0 * 16.0 ** 2))
    f.rho = f.rho + pulse
    target = 1.0 + 0.01 * sinusoids(n, n, rng(4, 1))
    return f, target


def vortex(n: int, radius: float, mach_v: float, mach_a: float, T_inf: float = 1.0,
           rho_inf: float = 1.0, angle: float = 0.0) -> Fields:
    """Isentropic vortex centred in an n x n periodic box.  Radial balance
    dp/dr = rho u_phi^2 / r with p = rho T and p ~ rho^gamma (gamma = 2) gives
    T = T_inf (1 - Ma_v^2 e^{1-r^2} / 2) and rho = rho_inf T / T_inf."""
    X, Y = _grid(n, n)
    c = np.sqrt(2.0 * T_inf)
    dx = X - n / 2.0
    dy = Y - n / 2.0
    r = np.hypot(dx, dy) / radius
    e = np.exp(0.5 * (1.0 - r * r))
    uphi = mach_v * c * r * e
    rr = np.maximum(np.hypot(dx, dy), 1e-300)
    U = mach_a * c
    ux = -uphi * dy / rr + U * np.cos(angle)
    uy = uphi * dx / rr + U * np.sin(angle)
    T = T_inf * (1.0 - 0.5 * mach_v * mach_v * e * e)
    return Fields(rho_inf * T / T_inf, ux, uy, T)


def ensemble_sizes(count: int = 256, lo: int = 32, hi: int = 512, seed_sub: int = 0):
    g = rng(5, seed_sub)
    nx = g.integers(lo, hi + 1, size=count)
    ny = g.integers(lo, hi + 1, size=count)
    return [int(v) for v in nx], [int(v) for v in ny]


def ensemble_member(i: int, nx: int, ny: int) -> Fields:
    g = rng(5, 1000 + i)
    M = g.uniform(0.0, 3.0)
    phi = g.uniform(0.0, 2.0 * np.pi)
    r = g.uniform(0.5, 4.0)
    rho = 1.0 + (0.1 / 8.0) * sinusoids(nx, ny, g, kmax=2)
    s = sinusoids(nx, ny, g, kmax=2)
    s = (s - s.min()) / max(s.max() - s.min(), 1e-300)
    T = 1.0 + (r - 1.0) * s
    return Fields(rho, np.full((ny, nx), M * np.cos(phi)), np.full((ny, nx), M * np.sin(phi)), T)


def ensemble(count: int = 256, lo: int = 32, hi: int = 512):
    nxs, nys = ensemble_sizes(count, lo, hi)
    return [ensemble_member(i, nxs[i], nys[i]) for i in range(count)]
