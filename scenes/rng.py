"""Counter-based SplitMix64 random stream for seeded synthetic scenes.

SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): the i-th output (i = 1, 2, ...) is the 64-bit
finaliser applied to ``seed + i * 0x9E3779B97F4A7C15`` (mod 2**64).  Uniforms
take the top 53 bits; Gaussians use the Box-Muller transform in float64.

This module draws scene inputs only; it contains none of the planner's
arithmetic.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, n: int) -> np.ndarray:
    """Outputs number ``start+1 .. start+n`` of the SplitMix64 sequence for ``seed``."""
    i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Stream:
    """Sequential view of one seed's SplitMix64 sequence."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.pos = 0

    def bits(self, n: int) -> np.ndarray:
        out = splitmix64(self.seed, self.pos, n)
        self.pos += n
        return out

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """U[lo, hi) in float64 from the top 53 bits."""
        u = (self.bits(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Uniform integers in the closed range [lo, hi]."""
        span = hi - lo + 1
        return lo + np.minimum((self.uniform(n) * span).astype(np.int64), span - 1)

    def normal(self, n: int) -> np.ndarray:
        """Standard normals by Box-Muller (cosine branch only)."""
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)

    def scalar(self) -> float:
        return float(self.uniform(1)[0])
