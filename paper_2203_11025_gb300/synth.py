"""Seeded synthetic inputs for the Helmholtz solver (media, right-hand sides).

This module holds none of the solver's arithmetic: it only produces inputs.
It is the one module shared by the CUDA path's tests/benchmark and the CPU
oracle, so both sides see bit-identical media and right-hand sides.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state_i = seed + (i+1)*golden,
then the published 64-bit finaliser.  Normals use the Box-Muller transform.

Media stand in for the paper's CIFAR-10-derived slowness models (Sec. 3.4.1):
a smoothed random image normalised to a fixed range.  Here the image is i.i.d.
N(0,1) noise filtered by a Gaussian (sigma = 8 cells, truncated at 4 sigma,
reflecting edges) and min-max mapped so that the slowness kappa lies in
[kappa_min, 1]; the solver consumes kappa^2 as float32.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """`count` outputs of SplitMix64 for stream `seed`, starting at counter `offset`."""
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in (0, 1): top 53 bits, shifted by half an ulp."""
    z = splitmix64(seed, count, offset)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller over consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:count]


def complex_normal(seed: int, shape) -> np.ndarray:
    """Complex standard normal: re and im i.i.d. N(0, 1/2)."""
    n = int(np.prod(shape))
    z = normal(seed, 2 * n) * np.sqrt(0.5)
    return (z[0::2] + 1j * z[1::2]).reshape(shape)


def grf_kappa2(ny: int, nx: int, seed: int, sigma: float = 8.0,
               kappa_min: float = 0.25, kappa_max: float = 1.0) -> np.ndarray:
    """Gaussian-random-field slowness medium; returns kappa^2 as float32 (ny, nx)."""
    from scipy.ndimage import gaussian_filter

    img = normal(seed, ny * nx).reshape(ny, nx)
    img = gaussian_filter(img, sigma=sigma, truncate=4.0, mode="reflect")
    lo, hi = img.min(), img.max()
    kappa = kappa_min + (kappa_max - kappa_min) * (img - lo) / (hi - lo)
    return (kappa * kappa).astype(np.float32)


def omega_for(n: int, kappa_max: float = 1.0, ppw: float = 10.0) -> float:
    """Angular frequency with max(omega*kappa*h) = 2*pi/ppw on an n-point grid, h = 1/n."""
    return 2.0 * np.pi / ppw * n / kappa_max


def source_positions(ny: int, nx: int, count: int, seed: int, margin: int):
    """`count` random interior nodes (iy, ix) at least `margin` cells from every edge."""
    u = uniform01(seed, 2 * count)
    iy = margin + np.floor(u[0::2] * (ny - 2 * margin)).astype(np.int64)
    ix = margin + np.floor(u[1::2] * (nx - 2 * margin)).astype(np.int64)
    return list(zip(iy.tolist(), ix.tolist()))


def point_sources(ny: int, nx: int, positions, h: float) -> np.ndarray:
    """One right-hand side per position: a unit point source, value 1/h^2 at the node."""
    g = np.zeros((len(positions), ny, nx), dtype=np.complex128)
    for k, (iy, ix) in enumerate(positions):
        g[k, iy, ix] = 1.0 / (h * h)
    return g


def gaussian_rhs(ny: int, nx: int, count: int, seed: int) -> np.ndarray:
    """`count` complex Gaussian random right-hand sides (i.i.d. per node)."""
    return complex_normal(seed, (count, ny, nx))


def pair_draws(seed: int, count: int, ny: int, nx: int, kmax: int):
    """Random numbers of the training-pair generator (Eq. 3.8-3.9), in the counter
    layout both implementations use: pair j's x ~ CN(0,1) is complex_normal of stream
    seed + 1 + j; its iteration count is k_j = 1 + floor(U_j kmax), U_j the j-th
    uniform of stream seed."""
    x = np.stack([complex_normal(seed + 1 + j, (ny, nx)) for j in range(count)])
    u = uniform01(seed, count)
    ks = np.minimum(1 + np.floor(u * kmax).astype(np.int64), kmax)
    return x, ks


def medium_seed(problem_id: int) -> int:
    return 1000 + problem_id


def rhs_seed(rhs_id: int) -> int:
    return 2000 + rhs_id
