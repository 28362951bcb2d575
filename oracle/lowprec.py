"""Rounding to bfloat16 for the oracle's low-precision pins (TEST INFRASTRUCTURE ONLY).

bfloat16 keeps the sign, the 8 exponent bits of binary32 and 8 significant bits
(7 stored).  Rounding a double to it (round to nearest, ties to even) is, for
values in the normal range of binary32, rounding the significand to 8 bits:
x = f * 2^e with f in [0.5, 1); f * 2^8 rounded half-to-even; times 2^(e-8).
Values below the binary32 normal range (|x| < 2^-126) become signed zero.

Split operands (the BF16X3 product): x = hi + lo + r with hi = bf16(x) and
lo = bf16(x - hi); the product A B is approximated by Ah Bh + Ah Bl + Al Bh,
leaving out Al Bl and the remainders (relative size about 2^-16).
"""
from __future__ import annotations

import numpy as np


def round_bf16(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    f, e = np.frexp(x)
    r = np.ldexp(np.rint(f * 256.0), e - 8)
    return np.where(np.abs(x) < 2.0 ** -126, 0.0 * x, r)


def split_bf16(x: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """hi = bf16(x), lo = bf16(x - hi)."""
    x = np.asarray(x, dtype=np.float64)
    hi = round_bf16(x)
    return hi, round_bf16(x - hi)
