"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the method: only the random-number generator and the
recipes that turn it into right-hand sides, initial blocks and system sizes.

Generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014).  State_i = seed + (i+1)*0x9E3779B97F4A7C15 (mod 2^64), output
= the mix64 finaliser of the state.  Uniform on [-1, 1): ((z >> 11) * 2^-53) * 2 - 1.
Gaussian: Box-Muller on two consecutive uniforms on (0, 1].
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """The n outputs of SplitMix64 seeded with `seed`, starting after `offset` draws."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed % (1 << 64)) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform on [0, 1) with 53 random bits."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform on [-1, 1)."""
    return uniform01(seed, n, offset) * 2.0 - 1.0


def gaussian(seed: int, n: int) -> np.ndarray:
    """Standard normal samples by Box-Muller on pairs of uniforms."""
    m = (n + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:n]


def rhs(nx: int, ny: int, nz: int, seed: int = 0) -> np.ndarray:
    """Right-hand side b ~ U[-1, 1) on the nx x ny x nz interior grid, shaped (nz, ny, nx)."""
    return uniform_pm1(seed, nx * ny * nz).reshape(nz, ny, nx)


def initial_block(nx: int, ny: int, nz: int, m: int, seed: int = 7) -> np.ndarray:
    """LOBPCG initial block X0: N x m Gaussian, column-major (shape (m, N) row-major)."""
    n = nx * ny * nz
    return gaussian(seed, n * m).reshape(m, n)


def uneven_dims(nsys: int, lo: int = 32, hi: int = 96, seed: int = 1000) -> np.ndarray:
    """Grid sides for `nsys` independent systems, i.i.d. uniform integers in [lo, hi] per axis.

    System i draws its three sides from its own stream seeded with seed + i."""
    out = np.zeros((nsys, 3), dtype=np.int64)
    for i in range(nsys):
        z = splitmix64(seed + i, 3)
        out[i] = lo + (z % np.uint64(hi - lo + 1)).astype(np.int64)
    return out


def net_init_weights(seed: int = 77, last_scale: float = 0.1) -> np.ndarray:
    """Initial weights of the learned post-correction (7776 values in the layout of the C ABI:
    [16][1][27], [16][16][27], [1][16][27]): Gaussian with standard deviation sqrt(2 / fan_in)
    (fan_in = input channels x 27), the last layer scaled by `last_scale` so that training starts
    near a zero correction."""
    g = gaussian(seed, 16 * 27 + 16 * 16 * 27 + 16 * 27)
    w1 = g[: 16 * 27] * np.sqrt(2.0 / 27)
    w2 = g[16 * 27: 16 * 27 + 16 * 16 * 27] * np.sqrt(2.0 / (16 * 27))
    w3 = g[16 * 27 + 16 * 16 * 27:] * np.sqrt(2.0 / (16 * 27)) * last_scale
    return np.concatenate([w1, w2, w3])
