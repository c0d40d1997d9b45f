"""Counter-based random numbers for synthetic traffic (splitmix64).

splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): the i-th output of stream s is mix(s + (i+1)*phi)
with phi = 0x9E3779B97F4A7C15 and mix the two xor-shift-multiply rounds below.
Being counter based, any draw can be regenerated on its own, which lets a
workload be rebuilt in chunks.
"""
from __future__ import annotations

import numpy as np

PHI = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
MASK53 = np.uint64((1 << 53) - 1)


def mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
    return z ^ (z >> np.uint64(31))


def derive(seed: int, *keys: int) -> int:
    """A stream id from a seed and integer keys (each key folded through mix64)."""
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for k in keys:
            s = mix64(s + PHI * np.uint64((int(k) + 1) & 0xFFFFFFFFFFFFFFFF))
    return int(s)


class Rng:
    """Sequential view of one splitmix64 stream; every call advances a counter."""

    def __init__(self, seed: int, *keys: int):
        self.stream = np.uint64(derive(seed, *keys))
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        i = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            return mix64(self.stream + i * PHI)

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) from the top 53 bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Integers uniform in [lo, hi] (inclusive), by scaling a uniform double."""
        span = hi - lo + 1
        v = np.floor(self.uniform(n) * span).astype(np.int64)
        return lo + np.minimum(v, span - 1)

    def normal(self, n: int) -> np.ndarray:
        """Standard normal doubles by the Box-Muller transform."""
        m = (n + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log1p(-u1))
        z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
        return z[:n]

    def log_uniform(self, lo: float, hi: float, n: int) -> np.ndarray:
        return np.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * self.uniform(n))

    def permutation(self, n: int) -> np.ndarray:
        return np.argsort(self.u64(n), kind="stable")

    def bytes(self, n: int) -> np.ndarray:
        w = self.u64((n + 7) // 8)
        return w.view(np.uint8)[:n].copy()
