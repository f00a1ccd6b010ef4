"""Seeded synthetic particle sets shared by the CUDA path's tests/bench and the oracle.

This module draws random numbers and shapes them into particle distributions; it
holds none of the FMM's arithmetic.  Every value comes from SplitMix64 (Steele,
Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):

    state += 0x9E3779B97F4A7C15
    z = (state ^ (state >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    out = z ^ (z >> 31)

The k-th output (k = 1, 2, ...) of a stream seeded with ``seed`` is therefore a
pure function of ``seed + k * 0x9E3779B97F4A7C15`` and is computed vectorised.
A uniform double in [0, 1) is the top 53 bits times 2**-53.  Points are
generated in float64 and rounded once to float32; the oracle consumes the same
float32 values promoted to float64, so the two sides differ only in arithmetic.

Distributions (the workloads of the paper's Results section, which places
particles "randomly in a cube" and "on a spherical shell", plus the Plummer
sphere used for adaptive trees):
  * ``uniform_cube``   x ~ U[0,1)^3, charges ~ U[-1,1].
  * ``plummer``        Plummer sphere, scale radius 1, truncated at r = 20 by
                       inverting the enclosed-mass fraction M(r) = r^3/(1+r^2)^1.5;
                       isotropic directions; equal charges 1/N.
  * ``sphere_shell``   uniform on the unit sphere surface, charges ~ U[-1,1].
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs ``start+1 .. start+n`` of the SplitMix64 stream seeded with ``seed``."""
    k = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, start: int = 0) -> np.ndarray:
    """n float64 values in [0, 1) from the top 53 bits of SplitMix64 outputs."""
    return (splitmix64(seed, n, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_cube(n: int, seed: int):
    """n points i.i.d. uniform in [0,1)^3, charges uniform in [-1,1]."""
    u = uniform01(seed, 4 * n)
    xyz = u[: 3 * n].reshape(n, 3).astype(np.float32)
    q = (2.0 * u[3 * n:] - 1.0).astype(np.float32)
    return np.ascontiguousarray(xyz), np.ascontiguousarray(q)


def plummer(n: int, seed: int, rmax: float = 20.0, equal_charges: bool = True):
    """Plummer sphere (scale radius 1) truncated at ``rmax``.

    Radius by inverse transform of the enclosed-mass fraction
    M(r) = r^3 / (1 + r^2)^(3/2):  X ~ U(0, M(rmax)),  r = (X^(-2/3) - 1)^(-1/2).
    Direction uniform on the sphere: cos(polar) ~ U[-1, 1], azimuth ~ U[0, 2*pi).
    Charges are 1/n each (or U[-1,1] when ``equal_charges`` is False).
    """
    u = uniform01(seed, 4 * n)
    mmax = rmax ** 3 / (1.0 + rmax * rmax) ** 1.5
    X = u[:n] * mmax
    X = np.maximum(X, 1e-300)
    r = 1.0 / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    cz = 2.0 * u[n: 2 * n] - 1.0
    az = 2.0 * math.pi * u[2 * n: 3 * n]
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    xyz = np.stack([r * sz * np.cos(az), r * sz * np.sin(az), r * cz], axis=1).astype(np.float32)
    if equal_charges:
        q = np.full(n, 1.0 / n, dtype=np.float32)
    else:
        q = (2.0 * u[3 * n:] - 1.0).astype(np.float32)
    return np.ascontiguousarray(xyz), np.ascontiguousarray(q)


def sphere_shell(n: int, seed: int):
    """n points uniform on the unit sphere surface, charges U[-1,1]."""
    u = uniform01(seed, 3 * n)
    cz = 2.0 * u[:n] - 1.0
    az = 2.0 * math.pi * u[n: 2 * n]
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    xyz = np.stack([sz * np.cos(az), sz * np.sin(az), cz], axis=1).astype(np.float32)
    q = (2.0 * u[2 * n:] - 1.0).astype(np.float32)
    return np.ascontiguousarray(xyz), np.ascontiguousarray(q)


def sample_indices(n: int, count: int, seed: int) -> np.ndarray:
    """``count`` distinct indices in [0, n), drawn by SplitMix64, sorted."""
    if count >= n:
        return np.arange(n, dtype=np.int64)
    picked: dict[int, None] = {}
    start = 0
    while len(picked) < count:
        draw = (splitmix64(seed, 2 * count, start) % np.uint64(n)).astype(np.int64)
        start += 2 * count
        for v in draw.tolist():
            if len(picked) < count:
                picked.setdefault(v, None)
    return np.array(sorted(picked), dtype=np.int64)


# The five workloads, with the sizes, distributions and parameters they are
# quoted on.  Config k draws from seed 1000 + k.
WORKLOADS = {
    "uniform4k": dict(kind="uniform", n=4096, p=4, theta=0.5, ncrit=64, max_depth=21, seed=1001),
    "uniform1m": dict(kind="uniform", n=1_048_576, p=10, theta=0.4, ncrit=64, max_depth=10, seed=1002),
    "plummer4m": dict(kind="plummer", n=4_194_304, p=8, theta=0.4, ncrit=64, max_depth=21, seed=1003),
    "batched512": dict(kind="batched", nsys=512, p=8, theta=0.5, ncrit=64, max_depth=21, seed=1004),
    "plummer16m": dict(kind="plummer", n=16_777_216, p=10, theta=0.4, ncrit=64, max_depth=21, seed=1005),
    # a quarter-size uniform case with the same p/theta/ncrit, for profiler captures
    "uniform262k": dict(kind="uniform", n=262_144, p=10, theta=0.4, ncrit=64, max_depth=10, seed=1006),
    # the paper's adaptive test: random points on a spherical shell, N_crit = 20,
    # FMM and hybrid at p = 8 (Results section, Fig. "cpu" C)
    "shell100k": dict(kind="shell", n=100_000, p=8, theta=0.5, ncrit=20, max_depth=21, seed=1007),
    "shell1m": dict(kind="shell", n=1_000_000, p=8, theta=0.5, ncrit=20, max_depth=21, seed=1008),
}


def make(kind: str, n: int, seed: int):
    if kind == "uniform":
        return uniform_cube(n, seed)
    if kind == "plummer":
        return plummer(n, seed)
    if kind == "shell":
        return sphere_shell(n, seed)
    raise ValueError(f"unknown distribution {kind!r}")


def batched_systems(nsys: int, seed: int, nmin: float = 1e3, nmax: float = 1e5):
    """Independent systems of log-uniform size; first half uniform cube, second half Plummer
    (charges U[-1,1] for both).  Returns (xyz, q, offsets) with offsets[nsys] = total."""
    u = uniform01(seed, nsys)
    sizes = np.rint(np.exp(math.log(nmin) + u * (math.log(nmax) - math.log(nmin)))).astype(np.int64)
    xs, qs = [], []
    for i, ni in enumerate(sizes.tolist()):
        if i < nsys // 2:
            x, q = uniform_cube(ni, seed * 7919 + i)
        else:
            x, q = plummer(ni, seed * 7919 + i, equal_charges=False)
        xs.append(x)
        qs.append(q)
    offsets = np.zeros(nsys + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    return np.concatenate(xs), np.concatenate(qs), offsets
