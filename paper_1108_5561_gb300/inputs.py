"""Seeded synthetic initial energy densities (GeV/fm^3) for the lattice
Boltzmann runs.  Holds no arithmetic of the method: it only draws hotspot
positions and amplitudes and sums Gaussians on the grid.

Recipe (both the CUDA path and the oracle receive these arrays):
  - smooth:  eps = eps0 exp(-r^2 / (2 sigma^2)) + floor, r from the grid centre,
    floor = 0.005 GeV/fm^3 (about eps(T = 0.1 GeV) for the crossover EOS)
  - hotspots: n Gaussians of width 0.4 fm, amplitudes ~ Exp(mean 20 GeV/fm^3),
    centres ~ N(0, 3 fm) per coordinate, on a uniform background of
    10 GeV/fm^3 (T about 0.3 GeV), sampled on a 0.1 fm grid
Random numbers come from splitmix64 with a Box-Muller transform so the draws
are identical on every machine.
"""
from __future__ import annotations

import math

import numpy as np

EPS_FLOOR = 0.005
HOTSPOT_BACKGROUND = 10.0
MASK = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.s = seed & MASK

    def next(self) -> int:
        self.s = (self.s + 0x9E3779B97F4A7C15) & MASK
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:  # (0, 1)
        return ((self.next() >> 11) + 0.5) / float(1 << 53)

    def normal(self) -> float:
        u1, u2 = self.uniform(), self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)

    def exponential(self, mean: float) -> float:
        return -mean * math.log(self.uniform())


def coords(nx: int, ny: int, dx: float):
    x = (np.arange(nx) - 0.5 * (nx - 1)) * dx
    y = (np.arange(ny) - 0.5 * (ny - 1)) * dx
    return np.meshgrid(x, y, indexing="xy")  # arrays of shape (ny, nx)


def smooth_gaussian(nx: int, ny: int, dx: float = 0.2, eps0: float = 30.0, sigma: float = 2.0,
                    floor: float = EPS_FLOOR) -> np.ndarray:
    X, Y = coords(nx, ny, dx)
    return eps0 * np.exp(-(X * X + Y * Y) / (2 * sigma * sigma)) + floor


def hotspots(nx: int, ny: int, dx: float = 0.1, n: int = 40, seed: int = 1108, width: float = 0.4,
             mean_amp: float = 20.0, spread: float = 3.0, floor: float = HOTSPOT_BACKGROUND):
    """Returns (eps, amplitudes, centres)."""
    rng = SplitMix64(seed)
    amps = np.array([rng.exponential(mean_amp) for _ in range(n)])
    cen = np.array([[spread * rng.normal(), spread * rng.normal()] for _ in range(n)])
    X, Y = coords(nx, ny, dx)
    eps = np.full((ny, nx), floor)
    for a, (cx, cy) in zip(amps, cen):
        eps += a * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * width * width))
    return eps, amps, cen


def batch_events(n: int = 512, seed: int = 1108, n_min: int = 64, n_max: int = 192,
                 eta_min: float = 0.04, eta_max: float = 0.3):
    """Events of a batch: square grids with side uniform in {n_min..n_max} and
    eta/s uniform in (eta_min, eta_max); returns [(side, eta/s), ...]."""
    r = SplitMix64(seed)
    out = []
    for _ in range(n):
        side = n_min + min(int(r.uniform() * (n_max - n_min + 1)), n_max - n_min)
        out.append((side, eta_min + (eta_max - eta_min) * r.uniform()))
    return out


def hotspot_basis(nx: int, ny: int, centres, dx: float = 0.1, width: float = 0.4):
    """The unit Gaussians of hotspots at `centres`, one row per hotspot, sites in
    storage order (row-major): eps0 = floor + amplitudes @ basis."""
    X, Y = coords(nx, ny, dx)
    return np.stack([np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * width * width)).reshape(-1)
                     for cx, cy in centres])
