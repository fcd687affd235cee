"""Pins for the compensated sums of Section 4 (Code 1 sum_3op, Code 2 sum_6op).

The defining property is the error-free transformation a + b = s + t in exact
arithmetic (sum_3op only when |a| >= |b|). Halves, their sums and the pairs
(s, t) are all exact in binary64, so the identity is checked exactly.
"""
import numpy as np
import pytest

import oracle as O


def _finite_halves():
    h = np.arange(0x10000, dtype=np.uint32).astype(np.uint16).view(np.float16)
    return h[np.isfinite(h)].astype(np.float64)


def _pairs(seed, nb=300):
    a = _finite_halves()
    rng = np.random.default_rng(seed)
    b = rng.choice(a, nb, replace=False)
    return np.repeat(a, b.size), np.tile(b, a.size)


def test_sum_6op_error_free_all_orders(oracle_lib):
    A, B = _pairs(10)
    s, t = O.compensated_sum(6, A, B, O.FP16)
    # no overflow of the rounded sum, nor of the intermediate s - b (TwoSum's
    # known overflow when |a| is near the largest half)
    ok = (np.abs(A + B) <= 65504.0) & np.isfinite(s) & (np.abs(s - B) <= 65504.0)
    assert ok.sum() > 10_000_000
    assert np.array_equal((A + B)[ok], (s + t)[ok])
    # s is the rounded sum
    assert np.array_equal(s[ok], O.round_to(A + B, O.FP16)[ok])


def test_sum_3op_error_free_when_ordered(oracle_lib):
    A, B = _pairs(11)
    s, t = O.compensated_sum(3, A, B, O.FP16)
    ok = (np.abs(A) >= np.abs(B)) & np.isfinite(s) & (np.abs(A + B) <= 65504.0)
    assert np.array_equal((A + B)[ok], (s + t)[ok])
    # and it is NOT error free in general when |a| < |b| (Section 4)
    bad = (np.abs(A) < np.abs(B)) & np.isfinite(s)
    assert np.any((A + B)[bad] != (s + t)[bad])


def test_sum_3op_6op_agree_when_ordered(oracle_lib):
    A, B = _pairs(12, nb=100)
    s3, t3 = O.compensated_sum(3, A, B, O.FP16)
    s6, t6 = O.compensated_sum(6, A, B, O.FP16)
    ok = (np.abs(A) >= np.abs(B)) & np.isfinite(s3) & np.isfinite(t6)
    assert np.array_equal(s3[ok], s6[ok])
    assert np.array_equal(t3[ok] + 0.0, t6[ok] + 0.0)


def test_eft_bf16_and_fp32(oracle_lib):
    rng = np.random.default_rng(13)
    n = 500_000
    for fmt, spread in ((O.BF16, 12), (O.FP32, 8)):
        A = O.round_to(rng.standard_normal(n) * np.exp2(rng.integers(-spread, spread, n)), fmt)
        B = O.round_to(rng.standard_normal(n) * np.exp2(rng.integers(-spread, spread, n)), fmt)
        s, t = O.compensated_sum(6, A, B, fmt)
        assert np.array_equal(A + B, s + t)
        s3, t3 = O.compensated_sum(3, A, B, fmt)
        ok = np.abs(A) >= np.abs(B)
        assert np.array_equal((A + B)[ok], (s3 + t3)[ok])
