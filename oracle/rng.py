"""SplitMix64 counter-based generator (oracle side).

Test infrastructure only (see ``oracle/__init__``).

The paper draws one random vector: the right-hand side of the 10 GMRES
iterations that estimate the largest eigenvalue for the Chebyshev bounds
(Sec. 6).  Both the oracle and the CUDA library draw it from the same
published generator, implemented independently on each side: SplitMix64
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014; the finaliser constants of Vigna's reference version), used as
a counter-based hash: value i of stream ``seed`` is
    z = seed + (i + 1) * 0x9E3779B97F4A7C15            (mod 2^64)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    z =  z ^ (z >> 31)
and mapped to [-1, 1) as (z >> 11) * 2^-52 - 1 (exact in FP64).
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, count):
    """Raw 64-bit outputs 0..count-1 of the stream ``seed``."""
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed, count):
    """Values in [-1, 1): (z >> 11) * 2^-52 - 1."""
    z = splitmix64(seed, count)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -52) - 1.0
