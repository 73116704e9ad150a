"""SplitMix64 (Steele, Lea, Flood, OOPSLA 2014; Vigna's published constants) with Box-Muller normals.

Counter-based: output i of a stream with seed s is mix(s + (i + 1) * golden), so any slice of a
stream can be generated without the ones before it.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class SplitMix64:
    """A sequential SplitMix64 stream: uint64 words, uniforms in (0, 1], N(0, 1) normals."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.pos = 0

    def words(self, count: int) -> np.ndarray:
        i = np.arange(self.pos + 1, self.pos + 1 + count, dtype=np.uint64)
        self.pos += count
        with np.errstate(over="ignore"):
            return _mix(self.seed + i * _GOLDEN)

    def uniform(self, count: int) -> np.ndarray:
        """Uniforms on (0, 1]: the top 53 bits plus one, scaled by 2^-53."""
        w = self.words(count)
        return ((w >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)

    def normal(self, count: int) -> np.ndarray:
        """Standard normals by the Box-Muller transform (cosine branch only)."""
        u1 = self.uniform(count)
        u2 = self.uniform(count)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)

    def integers(self, count: int, high: int) -> np.ndarray:
        """Integers in [0, high) by multiply-shift of the top 32 bits (bias < 2^-32 * high)."""
        w = self.words(count) >> np.uint64(32)
        return ((w * np.uint64(high)) >> np.uint64(32)).astype(np.int64)
