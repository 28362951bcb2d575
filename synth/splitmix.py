"""Counter-based SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), vectorised over numpy.

SplitMix64 advances its state by the golden-ratio increment 0x9E3779B97F4A7C15 and
returns a bijective mix of the state.  Output number ``i`` (0-based) of the stream
seeded with ``s`` is therefore ``mix(s + (i + 1) * 0x9E3779B97F4A7C15)`` (mod 2**64),
so any element of a stream can be computed on its own.  All arithmetic wraps
modulo 2**64, which numpy's uint64 does natively.

This module only draws numbers; it holds none of the sign method's arithmetic.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix64(z: np.ndarray) -> np.ndarray:
    """The SplitMix64 finaliser (variant 13 of Stafford's mixers)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def raw(seed: int, counters: np.ndarray) -> np.ndarray:
    """uint64 output number ``counters`` (array of 0-based indices) of stream ``seed``."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * GOLDEN
    return mix64(state)


def uniform01(seed: int, counters: np.ndarray) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of the output times 2**-53."""
    return (raw(seed, counters) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_pm1(seed: int, counters: np.ndarray) -> np.ndarray:
    """Doubles in [-1, 1): 2*u - 1 with u from :func:`uniform01` (exact in binary64)."""
    return 2.0 * uniform01(seed, counters) - 1.0


def substream(seed: int, tag: int) -> int:
    """Seed of an independent sub-stream, derived by mixing (seed, tag)."""
    with np.errstate(over="ignore"):
        v = mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ mix64(np.uint64(tag) + GOLDEN))
    return int(v)
