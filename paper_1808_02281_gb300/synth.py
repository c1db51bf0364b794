"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module holds random numbers and workload shapes only -- none of the
method's arithmetic.  Links are NOT built here: each side turns the drawn
algebra parameters omega into SU(3) links with its own exponential
(U = exp(i omega.T), Eq. 18_1_29_3 of the paper).

Random numbers come from the counter form of SplitMix64 (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): the i-th
64-bit word of stream ``seed`` is mix(seed + (i+1) * 0x9E3779B97F4A7C15).
Normals use the Box-Muller transform on consecutive word pairs (cosine
branch only), so the values are the same on every machine and numpy version.

Draw order for a field of shape [V, 4, 8]: site (x fastest), then direction
mu = 0..3, then algebra index a = 0..7 -- normal number  (n*4 + mu)*8 + a.
Spinor fields [V, 4, 3] complex: site, Dirac index, colour, then real and
imaginary part -- normal number ((n*4 + alpha)*3 + a)*2 + (0 re, 1 im).
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def words(seed: int, start: int, count: int) -> np.ndarray:
    """64-bit words start .. start+count-1 of SplitMix64 stream ``seed``."""
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA)


def normals(seed: int, count: int, start: int = 0) -> np.ndarray:
    """``count`` standard normals (normal j uses words 2j and 2j+1)."""
    out = np.empty(count, dtype=np.float64)
    for lo in range(0, count, _CHUNK):
        n = min(_CHUNK, count - lo)
        w = words(seed, 2 * (start + lo), 2 * n)
        u1 = ((w[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
        u2 = (w[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        out[lo:lo + n] = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return out


def volume(dims) -> int:
    v = 1
    for d in dims:
        v *= int(d)
    return v


def omega(dims, sigma: float, seed: int) -> np.ndarray:
    """Algebra parameters w_a ~ N(0, sigma^2) of every link, float64 [V, 4, 8]."""
    V = volume(dims)
    return (sigma * normals(seed, V * 32)).reshape(V, 4, 8)


def momenta(dims, seed: int) -> np.ndarray:
    """Gaussian su(3) momenta p^a ~ N(0, 1), float64 [V, 4, 8]."""
    V = volume(dims)
    return normals(seed, V * 32).reshape(V, 4, 8)


def gauge_parameters(dims, seed: int, sigma: float = 1.0) -> np.ndarray:
    """Algebra parameters v_a ~ N(0, sigma^2) of a gauge rotation g_n, [V, 8]."""
    V = volume(dims)
    return (sigma * normals(seed, V * 8)).reshape(V, 8)


def spinor(dims, seed: int) -> np.ndarray:
    """Gaussian spinor field, real and imaginary parts ~ N(0, 1):
    float64 [V, 4, 3, 2] (site, Dirac index, colour, re/im)."""
    V = volume(dims)
    return normals(seed, V * 24).reshape(V, 4, 3, 2)


def sample_links(n_links: int, count: int, seed: int) -> np.ndarray:
    """``count`` distinct link indices (site*4 + mu) out of n_links, sorted."""
    count = min(count, n_links)
    keys = words(seed, 0, n_links)
    idx = np.argpartition(keys, count - 1)[:count] if count < n_links else np.arange(n_links)
    return np.sort(idx.astype(np.int64))


# The synthetic workloads: lattice (Lx, Ly, Lz, Lt), link spread sigma of
# w_a ~ N(0, sigma^2), tadpole factor u0, inverse coupling beta, seed.
WORKLOADS = {
    "4^4": dict(dims=(4, 4, 4, 4), sigma=0.5, u0=0.87, beta=6.0, seed=0),
    "16^3x32": dict(dims=(16, 16, 16, 32), sigma=0.15, u0=0.86, beta=6.0, seed=0),
    "32^3x64": dict(dims=(32, 32, 32, 64), sigma=0.3, u0=0.87, beta=6.0, seed=0),
    "48^3x96": dict(dims=(48, 48, 48, 96), sigma=0.3, u0=0.87, beta=6.0, seed=0),
}

# Uneven-volume batch: four lattices each of these sizes.
BATCH_DIMS = [(8, 8, 8, 8)] * 4 + [(12, 12, 12, 24)] * 4 + [(16, 16, 16, 32)] * 4 + \
    [(24, 24, 24, 48)] * 4
