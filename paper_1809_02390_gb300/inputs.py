"""Seeded synthetic inputs (initial density fields) shared by the CUDA path,
its tests and the oracle.

This module holds none of the method's arithmetic: only the shapes of the
initial conditions (tanh droplet / slab / ellipse profiles between two given
densities, uniform noise) and a counter-based random generator.  The
coexistence densities it interpolates between are passed in by the caller.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) evaluated at counter
``seed * 2^32 + index``; the top 53 bits give a double in [0, 1).
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """SplitMix64 output for each 64-bit counter value."""
    with np.errstate(over="ignore"):
        z = (counter.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles uniform in [0, 1) from stream ``seed``."""
    idx = np.arange(offset, offset + n, dtype=np.uint64) + (np.uint64(seed) << np.uint64(32))
    return (splitmix64(idx) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def droplet(nx: int, ny: int, radius: float, width: float, rho_g: float, rho_l: float,
            center: tuple[float, float] | None = None) -> np.ndarray:
    """Circular liquid droplet, tanh profile rho = mid - (rho_l - rho_g)/2 tanh(2 (r - R)/W),
    centred at node (nx/2, ny/2) unless given; shape (ny, nx)."""
    cx, cy = (nx / 2.0, ny / 2.0) if center is None else center
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    return 0.5 * (rho_l + rho_g) - 0.5 * (rho_l - rho_g) * np.tanh(2.0 * (r - radius) / width)


def ellipse(nx: int, ny: int, semi_x: float, semi_y: float, width: float, rho_g: float,
            rho_l: float, noise: float = 0.0, seed: int = 0) -> np.ndarray:
    """Elliptic droplet (semi-axes along x and y) with a tanh profile across the
    level set of the normalised radius, times (1 + noise * U[-1, 1])."""
    cx, cy = nx / 2.0, ny / 2.0
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    q = np.sqrt(((x - cx) / semi_x) ** 2 + ((y - cy) / semi_y) ** 2)
    d = (q - 1.0) * math.sqrt(semi_x * semi_y)  # approximate signed distance
    rho = 0.5 * (rho_l + rho_g) - 0.5 * (rho_l - rho_g) * np.tanh(2.0 * d / width)
    if noise:
        rho = rho * (1.0 + noise * (2.0 * uniform(seed, nx * ny).reshape(ny, nx) - 1.0))
    return rho


def slab(nx: int, ny: int, thickness: float, width: float, rho_g: float, rho_l: float,
         axis: int = 1) -> np.ndarray:
    """Flat liquid slab of the given thickness centred in the domain, with two
    tanh interfaces normal to x (axis=1) or y (axis=0); shape (ny, nx)."""
    n = nx if axis == 1 else ny
    s = np.arange(n, dtype=np.float64)
    d = np.abs(s - n / 2.0) - thickness / 2.0
    prof = 0.5 * (rho_l + rho_g) - 0.5 * (rho_l - rho_g) * np.tanh(2.0 * d / width)
    return np.broadcast_to(prof[None, :] if axis == 1 else prof[:, None], (ny, nx)).copy()


def spinodal(nx: int, ny: int, rho_mean: float, amplitude: float = 0.01, seed: int = 0) -> np.ndarray:
    """Uniform density with seeded uniform relative noise: rho_mean (1 + amplitude U[-1, 1])."""
    u = uniform(seed, nx * ny).reshape(ny, nx)
    return rho_mean * (1.0 + amplitude * (2.0 * u - 1.0))


def batch_specs(n: int = 256, seed: int = 0, side_min: int = 64, side_max: int = 1024,
                tr_range=(0.65, 0.95), w_range=(3.0, 8.0)) -> list[dict]:
    """Seeded descriptions of ``n`` independent lattices: side length log-uniform in
    [side_min, side_max] (rounded), reduced temperature and interface width
    uniform in their ranges, and a droplet or a slab by a fair coin."""
    u = uniform(seed, 4 * n).reshape(n, 4)
    out = []
    for k in range(n):
        side = int(round(math.exp(math.log(side_min) + u[k, 0] * (math.log(side_max) - math.log(side_min)))))
        out.append({
            "nx": side, "ny": side,
            "Tr": tr_range[0] + u[k, 1] * (tr_range[1] - tr_range[0]),
            "W": w_range[0] + u[k, 2] * (w_range[1] - w_range[0]),
            "shape": "droplet" if u[k, 3] < 0.5 else "slab",
        })
    return out
