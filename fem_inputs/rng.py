"""Counter-based SplitMix64 generator (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), vectorised with numpy.

Draw i of stream `seed` is mix(seed + (i + 1) * 0x9E3779B97F4A7C15), so any
draw can be produced independently of the others and the sequence is the
same on every machine (uint64 arithmetic wraps modulo 2^64).
"""

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Return draws offset..offset+count-1 of stream `seed` as uint64."""
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """53-bit doubles in [0, 1): the top 53 bits of each draw times 2^-53."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(seed: int, count: int, lo: float, hi: float, offset: int = 0) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, count, offset)


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normal draws by the Box-Muller transform: draw 2i and 2i+1 of
    the stream give u1, u2 and z_i = sqrt(-2 ln(1 - u1)) cos(2 pi u2)."""
    u = uniform01(seed, 2 * count).reshape(count, 2)
    return np.sqrt(-2.0 * np.log1p(-u[:, 0])) * np.cos(2.0 * np.pi * u[:, 1])


def permutation(seed: int, n: int) -> np.ndarray:
    """A seeded permutation of range(n): argsort of n uniform draws (ties are
    impossible in practice; a stable sort keeps it deterministic anyway)."""
    return np.argsort(uniform01(seed, n), kind="stable").astype(np.int64)
