"""Counter-based thermal noise of the oracle.

Methods, "Replica batching": thermal noise from a device-side counter-based
Philox generator keyed by (seed, replica-and-cell index, step), reused
identically by the predictor and corrector (Stratonovich); the thermal
field's standard deviation per component is (Results, replica-batched
engine) sigma = sqrt(2 alpha kB T / (mu0^2 Ms V gamma0 dt)).

Philox4x32-10 follows its published definition (Salmon, Moraes, Dror &
Shaw, SC'11): ten rounds of two 32x32->64 multiplies (multipliers
0xD2511F53, 0xCD9E8D57) with the Weyl key schedule (0x9E3779B9, 0xBB67AE85).
The paper names only "counter-based Philox"; the layout is the reading
taken here:
    key     = (lo32(seed_r), hi32(seed_r))
    counter = (cell index within the replica, lo32(step), hi32(step), 0)
    u_k     = ((x_k >> 8) + 1) * 2^-24   in (0, 1], exact in float32
    n0, n1  = sqrt(-2 ln u0) (cos 2 pi u1, sin 2 pi u1)
    n2      = sqrt(-2 ln u2) cos 2 pi u3        (Box-Muller)
    H_th    = sigma (n0, n1, n2)
seed_r = splitmix64(seed + r) when per-replica seeds are not given
(splitmix64 as published by Steele, Lea & Flood, OOPSLA'14).
"""
from __future__ import annotations

import numpy as np

from .constants import GAMMA0, KB, MU0

_M32 = np.uint64(0xFFFFFFFF)
_MUL0 = np.uint64(0xD2511F53)
_MUL1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10.  Inputs are integer arrays holding 32-bit
    values; returns four uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & _M32 for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _M32
    k1 = np.asarray(k1, dtype=np.uint64) & _M32
    for rnd in range(10):
        p0 = _MUL0 * c0           # < 2^64: exact in uint64
        p1 = _MUL1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _M32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _M32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
        k0 = (k0 + _W0) & _M32
        k1 = (k1 + _W1) & _M32
    return tuple(v.astype(np.uint32) for v in (c0, c1, c2, c3))


def splitmix64(x):
    """One splitmix64 output for state x (Python int arithmetic mod 2^64)."""
    M = (1 << 64) - 1
    z = (int(x) + 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def raw(seed: int, step: int, ncell: int):
    """Four uint32 outputs for every cell 0..ncell-1 at a given step."""
    seed = int(seed) & ((1 << 64) - 1)
    cell = np.arange(ncell, dtype=np.uint64)
    step = int(step)
    return philox4x32_10(cell, step & 0xFFFFFFFF, (step >> 32) & 0xFFFFFFFF, 0,
                         seed & 0xFFFFFFFF, seed >> 32)


def uniforms(x):
    """u = ((x >> 8) + 1) * 2^-24 in (0, 1]."""
    return ((np.asarray(x, dtype=np.uint64) >> np.uint64(8)).astype(np.float64) + 1.0) * 2.0 ** -24


def normals(seed: int, step: int, ncell: int) -> np.ndarray:
    """(3, ncell) standard normals by Box-Muller from one Philox block per cell."""
    x0, x1, x2, x3 = raw(seed, step, ncell)
    u0, u1, u2, u3 = (uniforms(v) for v in (x0, x1, x2, x3))
    r0 = np.sqrt(-2.0 * np.log(u0))
    r2 = np.sqrt(-2.0 * np.log(u2))
    return np.stack([r0 * np.cos(2 * np.pi * u1), r0 * np.sin(2 * np.pi * u1),
                     r2 * np.cos(2 * np.pi * u3)])


def thermal_field(p, T: float, dt: float, seed: int, step: int) -> np.ndarray:
    """H_th (3, nz, ny, nx) in A/m; zero where Ms = 0 or T = 0."""
    shape = p.shape
    n = int(np.prod(shape))
    if T <= 0.0:
        return np.zeros((3,) + shape)
    V = p.d[0] * p.d[1] * p.d[2]
    with np.errstate(divide="ignore", invalid="ignore"):
        sigma = np.where(p.Ms > 0,
                         np.sqrt(2.0 * p.alpha * KB * T / (MU0 ** 2 * np.where(p.Ms > 0, p.Ms, 1.0) * V * GAMMA0 * dt)),
                         0.0)
    g = normals(seed, step, n).reshape((3,) + shape)
    return sigma * g
