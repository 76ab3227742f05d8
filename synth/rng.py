"""SplitMix64 stream (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), vectorised with numpy.

The n-th output of a SplitMix64 generator with state s is mix(s + n * GOLDEN), so a
block of outputs can be produced in one shot.  Used only for *placing* synthetic
geometry and cameras; the lens samples of the method come from Philox (a separate,
counter-based generator implemented independently on each side).
"""

import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def _mix(z):
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


class SplitMix64:
    def __init__(self, seed: int):
        self.state = int(seed) & _M64

    def u64(self, n: int) -> np.ndarray:
        k = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            s = np.uint64(self.state) + k * np.uint64(GOLDEN)
        self.state = (self.state + n * GOLDEN) & _M64
        return _mix(s)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * u

    def normal(self, n: int) -> np.ndarray:
        """Box-Muller standard normals."""
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)

    def integers(self, n: int, hi: int) -> np.ndarray:
        return (self.u64(n) % np.uint64(hi)).astype(np.int64)
