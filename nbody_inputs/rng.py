"""Counter-based SplitMix64 streams (numpy, vectorised).

SplitMix64 is Steele, Lea & Flood, "Fast splittable pseudorandom number
generators" (OOPSLA 2014): the state advances by the golden-ratio increment
0x9E3779B97F4A7C15 and each output is the state passed through the
"mix13" finaliser.  Here the generator is used in counter mode: draw ``k`` of a
stream is ``mix(key + (k + 1) * GOLDEN)``, so any draw can be produced without
producing the ones before it, and a vectorised call gives the same numbers as a
scalar loop.

This module holds no N-body arithmetic.  It only turns (seed, stream, counter)
into uniform doubles; both the oracle tests and the GPU path receive the arrays
it produces.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM = np.uint64(0x632BE59BD9B4E019)


def mix64(z):
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def stream_key(seed: int, stream: int) -> np.uint64:
    """Key of sub-stream ``stream`` of ``seed`` (both non-negative ints)."""
    with np.errstate(over="ignore"):
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        t = np.uint64((stream + 1) & 0xFFFFFFFFFFFFFFFF)
        return mix64(np.array([s + t * _STREAM], dtype=np.uint64))[0]


def raw(key: np.uint64, counter) -> np.ndarray:
    """uint64 draws ``counter`` (array of non-negative ints) of the stream ``key``."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(key + (c + np.uint64(1)) * GOLDEN)


def uniform(key: np.uint64, counter) -> np.ndarray:
    """Uniform doubles in the open interval (0, 1): (top 53 bits + 1/2) / 2^53."""
    r = raw(key, counter) >> np.uint64(11)
    return (r.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)
