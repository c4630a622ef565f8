"""Counter-based SplitMix64 stream (Steele, Lea and Flood, 2014).

Output i of stream (seed, tag) is the SplitMix64 finaliser applied to
``key + (i + 1) * GAMMA`` where ``key`` mixes the seed and the tag.  Being
counter based, any slice of a stream can be produced without generating the
prefix, and the values do not depend on how the caller batches requests.
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


def _key(seed, tag):
    with np.errstate(over="ignore"):
        k = _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF))
        k = _mix(k ^ (np.uint64(tag & 0xFFFFFFFFFFFFFFFF) * GAMMA))
    return k


def splitmix64(seed, tag, n, start=0):
    """Return ``n`` uint64 outputs of stream ``(seed, tag)`` starting at counter ``start``."""
    key = _key(seed, tag)
    idx = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + idx * GAMMA)


def uniform(seed, tag, n, lo=0.0, hi=1.0, start=0):
    """Doubles in [lo, hi) built from the top 53 bits of each output."""
    z = splitmix64(seed, tag, n, start)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def randint(seed, tag, n, lo, hi, start=0):
    """Integers in [lo, hi] (inclusive), by scaling a 53-bit uniform."""
    u = uniform(seed, tag, n, 0.0, 1.0, start)
    return lo + np.minimum(np.floor(u * (hi - lo + 1)).astype(np.int64), hi - lo)
