"""Counter-based SplitMix64.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) advances a 64-bit state by the golden-ratio increment
and passes it through a two-multiply finaliser.  Output ``k`` of the stream that
starts at ``seed`` is therefore a pure function of ``seed + (k + 1) * gamma``,
which lets numpy draw a whole stream at once.
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed, counters):
    """Outputs ``counters`` (array of int) of the SplitMix64 stream seeded by ``seed``."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * GAMMA
    return _mix(state)


def uniform01(seed, counters):
    """Doubles in [0, 1) from the top 53 bits of each SplitMix64 output."""
    return (splitmix64(seed, counters) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(seed, n, lo, hi):
    """``n`` doubles uniform in [lo, hi) from stream ``seed`` (counters 0..n-1)."""
    return lo + (hi - lo) * uniform01(seed, np.arange(n, dtype=np.uint64))
