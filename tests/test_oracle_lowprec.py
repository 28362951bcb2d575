"""Pin of the oracle's bfloat16 rounding (no GPU)."""
import numpy as np

from oracle.lowprec import round_bf16, split_bf16


def test_exact_values_unchanged():
    v = np.array([0.0, 1.0, -2.0, 1.5, 1 + 2 ** -7, 3.0 * 2 ** -100])
    assert np.array_equal(round_bf16(v), v)


def test_ties_to_even_and_nearest():
    one = 1.0
    u = 2.0 ** -7                     # bf16 spacing at 1
    assert round_bf16(np.array([one + u / 2]))[0] == one           # tie -> even (1.0)
    assert round_bf16(np.array([one + 3 * u / 2]))[0] == one + 2 * u  # tie -> even (1 + 2u)
    assert round_bf16(np.array([one + u / 2 + 2 ** -30]))[0] == one + u
    assert round_bf16(np.array([-(one + u / 2 + 2 ** -30)]))[0] == -(one + u)


def test_relative_error_bound_and_idempotent():
    x = np.random.default_rng(0).standard_normal(10000) * 10.0 ** np.random.default_rng(1).integers(-20, 20, 10000)
    r = round_bf16(x)
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x))     # unit roundoff of an 8-bit significand
    assert np.array_equal(round_bf16(r), r)
    # 8 significant bits: r * 2^(7 - floor(log2|r|)) is an integer
    e = np.floor(np.log2(np.abs(r)))
    assert np.all(np.ldexp(r, (7 - e).astype(int)) == np.round(np.ldexp(r, (7 - e).astype(int))))


def test_tiny_values_flush():
    assert round_bf16(np.array([2.0 ** -127]))[0] == 0.0


def test_split_parts_and_error():
    rng = np.random.default_rng(2)
    x = rng.standard_normal(10000) * 10.0 ** rng.integers(-20, 20, 10000)
    hi, lo = split_bf16(x)
    # both parts are bfloat16 numbers, hi is the rounding of x, lo the rounding of the rest
    assert np.array_equal(round_bf16(hi), hi) and np.array_equal(round_bf16(lo), lo)
    assert np.array_equal(hi, round_bf16(x))
    assert np.all(np.abs(lo) <= 2.0 ** -8 * np.abs(x))
    # hi + lo has about 16 significant bits: |x - hi - lo| <= 2^-8 |x - hi| <= 2^-16 |x|
    assert np.all(np.abs(x - hi - lo) <= 2.0 ** -8 * np.abs(x - hi))
    assert np.all(np.abs(x - hi - lo) <= 2.0 ** -16 * np.abs(x))


def test_split_of_short_values_is_exact():
    # a value with at most 16 significant bits whose tail needs no rounding splits exactly
    v = np.array([1.0, 1 + 2 ** -7 + 2 ** -9, -(3 + 2 ** -12), 0.0, 2 ** -50 * (1 + 2 ** -15)])
    hi, lo = split_bf16(v)
    assert np.array_equal(hi + lo, v)
    assert split_bf16(np.array([1 + 2 ** -7]))[1][0] == 0.0
