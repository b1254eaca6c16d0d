"""SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), written from its published
definition: a Weyl sequence with increment 0x9E3779B97F4A7C15 followed by the
"mix13" finaliser.  Counter-based: output k of stream ``seed`` depends only on
(seed, k)."""

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, count, offset=0):
    """Outputs offset .. offset+count-1 of the SplitMix64 stream of ``seed``."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed, count, lo=0.0, hi=1.0, offset=0):
    """Doubles uniform in [lo, hi) from the top 53 bits of each output."""
    u = (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u
