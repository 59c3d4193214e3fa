"""Counter-based SplitMix64 generator for the seeded inlet noise.

ORACLE -- test infrastructure only.

The paper has no inlet noise; the channel workloads add a seeded 1 % uniform
perturbation to the inlet velocity.  It is drawn from SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the n-th output
(n = 0, 1, ...) for seed s is mix(s + (n + 1) * 0x9E3779B97F4A7C15 mod 2^64) with
mix(z) = z1 ^ (z1 >> 31), z1 = (z0 ^ (z0 >> 27)) * 0x94D049BB133111EB,
z0 = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9 (all mod 2^64).  A 64-bit output becomes a
double in [0, 1) from its top 53 bits, and xi = 2 u - 1 in [-1, 1).

The counter of the inlet node (y, z) at time step t (1-based) is n = (t * ny + y) * nz + z.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counter: np.ndarray) -> np.ndarray:
    """n-th SplitMix64 output for every n in ``counter`` (uint64 array)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counter.astype(np.uint64) + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, counter: np.ndarray) -> np.ndarray:
    """xi in [-1, 1) from the top 53 bits of the SplitMix64 output."""
    z = splitmix64(seed, counter)
    u01 = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u01 - 1.0


def inlet_noise(seed: int, t: int, ny: int, nz: int) -> np.ndarray:
    """xi(t, y, z) for every inlet node, shape (nz, ny)."""
    zz, yy = np.meshgrid(np.arange(nz, dtype=np.uint64), np.arange(ny, dtype=np.uint64), indexing="ij")
    with np.errstate(over="ignore"):
        counter = (np.uint64(t) * np.uint64(ny) + yy) * np.uint64(nz) + zz
    return uniform_pm1(seed, counter)
