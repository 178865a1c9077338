"""The compensated FP32 (double-float) list-order sum that the mixed-precision reductions use.

The device reductions add per-pair FP32 products with Knuth's TwoSum, keeping the rounding error of
each addition in a second FP32 word.  This checks the claim the design rests on, in numpy FP32
arithmetic with the same operation order: hi + lo matches the exact sum of the FP32 terms to about
2^-44 of the sum of their magnitudes (plain FP32 accumulation is off by ~2^-24 per term), i.e. as
close as an FP64 accumulation would be, for the term counts and cancellation of the List 2 and
List 3 far reductions.
"""
from fractions import Fraction

import numpy as np


def _df_sum(terms):
    f = np.float32
    hi, lo = f(0), f(0)
    for x in terms:
        x = f(x)
        t = f(hi + x)
        bp = f(t - hi)
        err = f(f(hi - f(t - bp)) + f(x - bp))
        hi = t
        lo = f(lo + err)
    return float(hi) + float(lo)


def _exact(terms):
    return float(sum(Fraction(float(np.float32(x))) for x in terms))


def test_double_float_sum_matches_the_exact_sum():
    rng = np.random.default_rng(7)
    for n, scale_spread in ((8, 1.0), (115, 1.0), (400, 6.0), (875, 3.0)):
        # magnitudes spread over several decades, mixed signs: heavy cancellation
        mags = 10.0 ** rng.uniform(-scale_spread, 0.0, n)
        terms = (mags * rng.choice([-1.0, 1.0], n)).astype(np.float32)
        exact = _exact(terms)
        bound = float(np.sum(np.abs(terms.astype(np.float64))))
        err_df = abs(_df_sum(terms) - exact)
        naive = np.float32(0)
        for x in terms:
            naive = np.float32(naive + x)
        err_naive = abs(float(naive) - exact)
        assert err_df <= 2.0 ** -44 * bound, (n, err_df / bound)
        assert err_df <= err_naive  # never worse than plain FP32 accumulation


def test_double_float_sum_is_exact_for_exactly_representable_partial_sums():
    terms = np.array([1.0, 2.0 ** -30, -1.0, 3.0, 2.0 ** -40], dtype=np.float32)
    assert _df_sum(terms) == 3.0 + 2.0 ** -30 + 2.0 ** -40
