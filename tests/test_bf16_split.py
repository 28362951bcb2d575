"""The split-BF16 operands of the tensor-core tier: the library's FP64 -> BF16 rounding (integer
operations on the IEEE-754 encoding) and its split x = hi + lo (hi = bf16(x), lo = bf16(x - hi)),
built for the host from the same header as the packing kernel, against the oracle's rounding
(round the significand to 8 bits, ties to even; below binary32's normal range signed zero), bit
for bit."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from oracle import lowprec

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("bf16") / "libbf16split.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I",
                    os.path.join(ROOT, "paper_2003_03868_gb300", "csrc"), "-o", out,
                    os.path.join(ROOT, "tests", "bf16_split_shim.cpp")], check=True)
    L = C.CDLL(out)
    p = C.c_void_p
    L.bf16_split_many.argtypes = [p, C.c_int64, p, p]
    L.bf16_round_many.argtypes = [p, C.c_int64, p]
    return L


def _bits(v):
    with np.errstate(over="ignore"):
        return (np.asarray(v, dtype=np.float64).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)


def _run(shim, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    hi = np.empty(x.size, dtype=np.uint16)
    lo = np.empty(x.size, dtype=np.uint16)
    rb = np.empty(x.size, dtype=np.uint16)
    shim.bf16_split_many(x.ctypes.data, x.size, hi.ctypes.data, lo.ctypes.data)
    shim.bf16_round_many(x.ctypes.data, x.size, rb.ctypes.data)
    return hi, lo, rb


def _inputs():
    g = np.random.default_rng(2003)
    u = g.integers(0, 2 ** 63, size=400_000, dtype=np.uint64) | (g.integers(0, 2, 400_000, dtype=np.uint64) << 63)
    x = u.view(np.float64)
    x = x[np.isfinite(x) & (np.abs(x) < 2.0 ** 127)]                  # every exponent of binary32's range and below
    x = x[np.abs(np.frexp(x)[1]) < 400] if x.size else x
    parts = [x, g.uniform(-2, 2, 200_000), g.uniform(-1, 1, 200_000) * 2.0 ** g.uniform(-140, 5, 200_000)]
    # significands at, just above and just below the rounding ties of hi and of lo, and carries
    m = g.integers(0, 2 ** 52, size=50_000, dtype=np.uint64)
    top = m & ~np.uint64(2 ** 45 - 1)
    for v in (top, top | np.uint64(2 ** 44), (top | np.uint64(2 ** 44)) + np.uint64(1),
              (top | np.uint64(2 ** 44)) - np.uint64(1), m | np.uint64(2 ** 44 - 1),
              (m & ~np.uint64(2 ** 37 - 1)) | np.uint64(2 ** 36), np.full(50_000, 2 ** 52 - 1, dtype=np.uint64)):
        e = g.integers(1023 - 130, 1023 + 127, size=v.size).astype(np.uint64)
        s = g.integers(0, 2, size=v.size).astype(np.uint64)
        parts.append(((s << np.uint64(63)) | (e << np.uint64(52)) | (v & np.uint64(2 ** 52 - 1))).view(np.float64))
    # ties of lo: x - hi = +-(q2 2^sh + 2^(sh-1)) ulps with q2 of 8 bits (odd and even), after a
    # hi rounded down (bit 44 clear) and after a hi rounded up (x - hi negative)
    q2 = g.integers(128, 256, size=50_000).astype(np.uint64)
    sh = g.integers(1, 37, size=50_000).astype(np.uint64)
    tie = (q2 << sh) | (np.uint64(1) << (sh - np.uint64(1)))
    for v in (top | tie, top | (np.uint64(2 ** 45) - tie)):
        e = g.integers(1023 - 100, 1023 + 100, size=v.size).astype(np.uint64)
        s = g.integers(0, 2, size=v.size).astype(np.uint64)
        parts.append(((s << np.uint64(63)) | (e << np.uint64(52)) | (v & np.uint64(2 ** 52 - 1))).view(np.float64))
    parts.append(np.array([0.0, -0.0, 1.0, -1.0, 2.0 ** -126, -(2.0 ** -126), 2.0 ** -127, np.nextafter(2.0 ** -126, 0),
                           3.3895313892515355e38, 3.3895313892515357e38, 5e-324, 1e-300, 1.0 + 2 ** -8, 1.0 + 2 ** -9]))
    return np.concatenate(parts)


def test_split_matches_the_rounding_definition_bit_for_bit(shim):
    x = _inputs()
    hi, lo, rb = _run(shim, x)
    ohi, olo = lowprec.split_bf16(x)
    assert np.array_equal(rb, _bits(lowprec.round_bf16(x)))
    assert np.array_equal(hi, _bits(ohi))
    assert np.array_equal(lo, _bits(olo))


def test_split_recovers_sixteen_bits(shim):
    # |x - hi - lo| <= 2^-16 |x| (about), and hi + lo is exact where the significand has <= 16 bits
    g = np.random.default_rng(2004)
    x = g.uniform(-1, 1, 100_000) * 2.0 ** g.uniform(-30, 30, 100_000)
    hi, lo, _ = _run(shim, x)
    val = lambda b: (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    assert np.all(np.abs(x - val(hi) - val(lo)) <= 2.0 ** -16 * np.abs(x))
    y = np.ldexp(np.floor(np.ldexp(x, 15 - np.frexp(x)[1])), np.frexp(x)[1] - 15)   # 15 significant bits
    hi, lo, _ = _run(shim, y)
    assert np.array_equal(val(hi) + val(lo), y)
