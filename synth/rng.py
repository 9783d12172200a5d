"""Counter-based random numbers from SplitMix64.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) produces its i-th output as mix(state0 + (i+1)*G)
with G = 0x9E3779B97F4A7C15 and the 64-bit finaliser
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9
    z ^= z >> 27; z *= 0x94D049BB133111EB
    z ^= z >> 31
so output i depends on (state0, i) alone.  Here state0 is a key derived from
(seed, stream) and i is a structured counter, which makes every draw
addressable without sequential state.  Doubles in [0, 1) take the top 53 bits.
"""
import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(state0, i):
    """The i-th SplitMix64 output (0-based) of the sequence seeded with state0."""
    state0 = np.asarray(state0, dtype=np.uint64)
    i = np.asarray(i, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = state0 + (i + np.uint64(1)) * _G
    return _mix(z)


def stream_key(seed, stream):
    """A 64-bit key for an independent sub-stream (seed, stream)."""
    k0 = splitmix64(np.uint64(seed), np.uint64(0))
    return splitmix64(k0, np.uint64(stream))


def uniform01(key, ctr):
    """Doubles uniform in [0, 1): the top 53 bits of output `ctr` of `key`."""
    z = splitmix64(key, ctr)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
