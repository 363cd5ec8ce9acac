"""Seeded synthetic inputs shared by the CPU oracle and the GPU path.

This module holds none of the method's arithmetic (no covariance, no
ordering, no factorisation): only a counter-based random generator, the
jittered-grid location recipe, standard-normal draws and the parameter walk
used to move theta between likelihood evaluations.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; constants as published by
Vigna).  splitmix64(s) below is the first output of a generator whose state
is s, i.e. mix(s + GAMMA).  Draw c of the stream keyed by `seed` is
splitmix64(splitmix64(seed) XOR c): a pure function of (seed, counter), so
the same inputs are produced on any host.

Location recipe (the paper draws its locations in the unit square, Sec. 5;
the workloads here use a perturbed regular grid):
  G = ceil(sqrt(n)), h = 1 / G, point p = j * G + i for the first n cells in
  row-major order (i fastest), x = (i + 0.5) h + (2 u1 - 1) 0.4 h,
  y = (j + 0.5) h + (2 u2 - 1) 0.4 h, with u1 = U(seed, 2p), u2 = U(seed, 2p+1).
Layout: one float64 array of length 2n, x[0..n) then y[0..n) (SoA).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(state: np.ndarray) -> np.ndarray:
    """First SplitMix64 output of a generator whose state is `state` (uint64 array)."""
    s = np.asarray(state, dtype=np.uint64)
    return _mix(s + GAMMA)


def stream_u64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """`count` uint64 draws (counters start..start+count) of the stream keyed by `seed`."""
    key = splitmix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
    ctr = np.arange(start, start + count, dtype=np.uint64)
    return splitmix64(key ^ ctr)


def uniform(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform float64 draws in [0, 1) with 53 random bits each."""
    v = stream_u64(seed, count, start) >> np.uint64(11)
    return v.astype(np.float64) * (1.0 / 9007199254740992.0)


def jittered_grid(n: int, seed: int = 1, jitter: float = 0.4) -> np.ndarray:
    """n locations of a perturbed G x G grid in (0,1)^2, SoA float64 of length 2n."""
    if n <= 0:
        return np.zeros(0, dtype=np.float64)
    g = int(math.isqrt(n - 1)) + 1 if n > 1 else 1
    h = 1.0 / g
    p = np.arange(n, dtype=np.int64)
    i = (p % g).astype(np.float64)
    j = (p // g).astype(np.float64)
    u = uniform(seed, 2 * n)
    u1 = u[0::2]
    u2 = u[1::2]
    x = (i + 0.5) * h + (2.0 * u1 - 1.0) * (jitter * h)
    y = (j + 0.5) * h + (2.0 * u2 - 1.0) * (jitter * h)
    return np.concatenate([x, y])


def standard_normal(n: int, seed: int = 2) -> np.ndarray:
    """n independent N(0,1) draws by the Box-Muller transform of uniform pairs."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    w = np.empty(2 * m, dtype=np.float64)
    w[0::2] = r * np.cos(2.0 * math.pi * u2)
    w[1::2] = r * np.sin(2.0 * math.pi * u2)
    return w[:n].copy()


def theta_walk(theta0, steps: int, seed: int = 7, scale: float = 0.05,
               lo=(0.05, 0.005, 0.2), hi=(20.0, 3.0, 4.0)) -> np.ndarray:
    """A fixed pseudo-random walk in log(sigma2, beta, nu) starting at theta0.

    Each step multiplies every parameter by exp(scale * (2u - 1)); values are
    clamped to [lo, hi].  Returns an array of shape (steps, 3).
    """
    t = np.log(np.asarray(theta0, dtype=np.float64))
    out = np.empty((steps, 3), dtype=np.float64)
    u = uniform(seed, 3 * steps).reshape(steps, 3)
    llo, lhi = np.log(lo), np.log(hi)
    for k in range(steps):
        out[k] = np.exp(t)
        t = np.clip(t + scale * (2.0 * u[k] - 1.0), llo, lhi)
    return out


def dataset(n: int, loc_seed: int = 1, z_seed: int = 2):
    """Locations (SoA, generation order) and the standard-normal vector w used to draw Z."""
    return jittered_grid(n, loc_seed), standard_normal(n, z_seed)
