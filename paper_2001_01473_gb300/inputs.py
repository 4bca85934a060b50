"""Seeded synthetic inputs for the stencil sweeps.

This module is shared by the CUDA path's tests, the benchmark and the CPU
oracle harness.  It holds random streams and workload recipes only: no
stencil arithmetic.  Every value is a deterministic function of a seed.

Random stream: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014).  Output k of stream `seed` is
mix(seed + (k+1) * 0x9E3779B97F4A7C15), so any slice of the stream can be
produced independently.  A uniform [0,1) value keeps the top `bits` bits:
24 for FP32/FP16 workloads (every value exactly representable in FP32),
53 for FP64 workloads.

Workloads follow the paper's methodology (Section 5.1: 16384^2 and 512^3 grids,
1000 iterations, single and double precision) and the synthetic benchmark
family of Table 4 (star/box stencils of radius 1-4 with constant
per-offset coefficients).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STAR = 0
BOX = 1


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs start..start+n-1 of the SplitMix64 stream seeded with `seed`."""
    with np.errstate(over="ignore"):
        k = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, bits: int = 53, start: int = 0) -> np.ndarray:
    """n uniform [0,1) doubles carrying the top `bits` bits of the stream."""
    if not 1 <= bits <= 53:
        raise ValueError("bits must be in [1, 53]")
    z = splitmix64(seed, n, start) >> np.uint64(64 - bits)
    return z.astype(np.float64) * (2.0 ** -bits)


def bits_for(dtype: str) -> int:
    """Mantissa bits drawn for a workload dtype (FP32/FP16 runs: 24, FP64: 53)."""
    return 53 if dtype == "f64" else 24


def npdtype(dtype: str):
    """numpy storage type of a workload dtype name."""
    return {"f32": np.float32, "f64": np.float64, "f16": np.float16,
            "f32c": np.float32}[dtype]


def coeff_count(ndim: int, shape: int, radius: int) -> int:
    """Points in a star (2*d*R+1) or box ((2R+1)^d) stencil (Table 4)."""
    if shape == STAR:
        return 2 * ndim * radius + 1
    return (2 * radius + 1) ** ndim


def padded_shape(dims, radius: int):
    """C-order extents of the padded array: interior + radius-wide halo per side."""
    return tuple(int(d) + 2 * radius for d in dims)


def normalised_coeffs(n: int, seed: int = 0) -> np.ndarray:
    """Raw uniform [0,1) FP64 coefficients divided by their FP64 sum.

    The sum is accumulated in index order k = 0..n-1 (the canonical offset
    order).  The caller rounds the result once to the run's dtype.
    """
    raw = uniform(seed, n, 53)
    s = 0.0
    for v in raw:
        s += float(v)
    return raw / s


def field(dims, radius: int, seed: int = 1, dtype: str = "f32") -> np.ndarray:
    """Uniform [0,1) field over the whole padded array (halo included)."""
    shp = padded_shape(dims, radius)
    n = int(np.prod(shp))
    return uniform(seed, n, bits_for(dtype)).reshape(shp).astype(npdtype(dtype))


def target_field(dims, radius: int, seed: int = 2, dtype: str = "f32") -> np.ndarray:
    """Loss target for the adjoint workload: uniform [0,1), padded shape."""
    return field(dims, radius, seed, dtype)


def heat_coeffs(ndim: int, a: float = 0.1) -> np.ndarray:
    """Explicit heat-diffusion star stencil, radius 1: centre 1-2*d*a, each neighbour a."""
    n = 2 * ndim + 1
    c = np.full(n, a, dtype=np.float64)
    c[0] = 1.0 - 2 * ndim * a
    return c


def gaussian_bump(dims, radius: int, seed: int = 1, dtype: str = "f32",
                  noise: float = 0.01) -> np.ndarray:
    """Centred Gaussian bump (sigma = n_i/8 per axis, amplitude 1) plus noise*U[0,1).

    Evaluated in FP64 over the padded array with coordinates of the interior
    (halo cells use the same formula), then converted to the storage dtype.
    """
    shp = padded_shape(dims, radius)
    grids = np.meshgrid(*[np.arange(s, dtype=np.float64) - radius for s in shp],
                        indexing="ij")
    e = np.zeros(shp, dtype=np.float64)
    for g, n in zip(grids, dims):
        c = (n - 1) / 2.0
        sig = n / 8.0
        e += (g - c) ** 2 / (2.0 * sig * sig)
    u = np.exp(-e)
    u += noise * uniform(seed, int(np.prod(shp)), 24).reshape(shp)
    return u.astype(npdtype(dtype))


@dataclass(frozen=True)
class GridDesc:
    """One grid of the batched workload."""
    ny: int
    nx: int
    shape: int
    radius: int
    T: int


def batch_descs(n: int = 512, seed: int = 3, side_lo: int = 128,
                side_hi: int = 4096, t_lo: int = 10, t_hi: int = 500) -> list:
    """Batched workload: n independent 2D grids.

    Side lengths are log-uniform in [side_lo, side_hi] per axis (so grids
    are not square), shape star/box and radius 1-2 drawn per grid, T
    uniform in [t_lo, t_hi].  Six draws per grid from one stream.
    """
    u = uniform(seed, 6 * n, 53).reshape(n, 6)
    lo, hi = math.log(side_lo), math.log(side_hi)
    out = []
    for i in range(n):
        ny = int(round(math.exp(lo + (hi - lo) * u[i, 0])))
        nx = int(round(math.exp(lo + (hi - lo) * u[i, 1])))
        shape = STAR if u[i, 2] < 0.5 else BOX
        radius = 1 if u[i, 3] < 0.5 else 2
        T = t_lo + int(u[i, 4] * (t_hi - t_lo + 1))
        out.append(GridDesc(ny, nx, shape, radius, T))
    return out
