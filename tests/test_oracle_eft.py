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


# ---------------------------------------------------------------------------
# The solution update as the solvers apply it (Algorithm 2 with R = T + inc;
# reading A5 for binary32 registers over half storage).
# ---------------------------------------------------------------------------

def _bf16_round(x):
    import torch
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _quantum(x, fmt):
    """Spacing of the storage format's values around |x| (the subnormal
    spacing below the smallest normal)."""
    p, emin = (11, -14) if fmt == O.FP16 else (8, -126)
    e = np.floor(np.log2(np.maximum(np.abs(x), np.ldexp(1.0, emin))))
    return np.ldexp(1.0, (e - (p - 1)).astype(int))


def _update_inputs(seed, fmt, n=400_000):
    """Stored V and T (T of the size of V's rounding, or arbitrary), binary32
    increments spread over many binades, and edge cases."""
    rng = np.random.default_rng(seed)
    rnd = (lambda x: np.asarray(x, np.float16).astype(np.float64)) if fmt == O.FP16 else _bf16_round
    V = rnd(rng.standard_normal(n) * np.exp2(rng.integers(-10, 8, n)))
    T = rnd(V * np.exp2(-12.0) * rng.uniform(-1, 1, n))
    T[: n // 8] = rnd(rng.standard_normal(n // 8) * np.exp2(rng.integers(-20, 2, n // 8)))
    inc = np.asarray(V * np.exp2(rng.integers(-30, 3, n).astype(float)) * rng.standard_normal(n),
                     np.float32).astype(np.float64)
    # edge cases: zeros, exact cancellation, subnormals, halfway sums
    k = n // 16
    V[:k] = 0.0
    inc[k:2 * k] = -V[k:2 * k]
    T[k:2 * k] = 0.0
    tiny = np.ldexp(1.0, -24) if fmt == O.FP16 else np.ldexp(1.0, -133)
    V[2 * k:3 * k] = rnd(tiny * rng.integers(-600, 600, k))
    inc[2 * k:3 * k] = np.asarray(tiny * rng.uniform(-900, 900, k), np.float32)
    inc[3 * k:4 * k] = 0.5 * _quantum(V[3 * k:4 * k], fmt) * np.sign(rng.standard_normal(k))
    T[3 * k:4 * k] = 0.0
    return V, T, inc


def _violations_f32(V, T, inc, Vo, To, fmt):
    """Properties of the binary32-register update, with s = V + (T + inc)
    evaluated in numpy's binary32 arithmetic: V' is the storage value nearest
    to s, and V' + T' represents s to within half a storage quantum of the
    residual s - V' (the one rounding A5 allows)."""
    f32 = np.float32
    s = (V.astype(f32) + (T.astype(f32) + inc.astype(f32))).astype(np.float64)
    rnd = (lambda x: np.asarray(x, np.float16).astype(np.float64)) if fmt == O.FP16 else _bf16_round
    bad_v = Vo != rnd(s)
    e = s - Vo                                    # exact in binary64
    bad_t = np.abs((Vo + To) - s) > 0.5 * _quantum(e, fmt)
    bad_t |= (To != 0) & (np.sign(To) != np.sign(e))
    return int(np.count_nonzero(bad_v | bad_t))


@pytest.mark.parametrize("fmt", [O.FP16, O.BF16])
def test_binary32_register_compensated_update(oracle_lib, fmt):
    V, T, inc = _update_inputs(20 + fmt, fmt)
    Vo, To = O.solution_update(3, V, T, inc, fmt, O.FP32)
    assert _violations_f32(V, T, inc, Vo, To, fmt) == 0
    # the residual carried in T' is not lost: V' + T' is closer to s than V'
    s = (V.astype(np.float32) + (T.astype(np.float32) + inc.astype(np.float32))).astype(np.float64)
    assert np.sum(np.abs(Vo + To - s)) < 0.05 * np.sum(np.abs(Vo - s))
    # planted mistakes (the oracle's own update fed what the mistake computes)
    Vd, Td = O.solution_update(3, V, np.zeros_like(T), inc, fmt, O.FP32)     # T dropped
    assert _violations_f32(V, T, inc, Vd, Td, fmt) > 1000
    Vn, Tn = O.solution_update(3, V, -T, inc, fmt, O.FP32)                    # T subtracted
    assert _violations_f32(V, T, inc, Vn, Tn, fmt) > 1000
    assert _violations_f32(V, T, inc, Vo, np.zeros_like(To), fmt) > 1000    # T' dropped
    assert _violations_f32(V, T, inc, Vo, -To, fmt) > 1000                  # T' negated


@pytest.mark.parametrize("fmt", [O.FP16, O.BF16])
def test_binary32_register_plain_update(oracle_lib, fmt):
    """Without compensation: V' = RN_storage(RN32(V + inc))."""
    V, T, inc = _update_inputs(30 + fmt, fmt)
    Vo, To = O.solution_update(0, V, T, inc, fmt, O.FP32)
    s = (V.astype(np.float32) + inc.astype(np.float32)).astype(np.float64)
    rnd = (lambda x: np.asarray(x, np.float16).astype(np.float64)) if fmt == O.FP16 else _bf16_round
    assert np.array_equal(Vo, rnd(s))
    assert np.array_equal(To, T)


@pytest.mark.parametrize("comp", [3, 6])
def test_half_compensated_update_carries_T(oracle_lib, comp):
    """Same format throughout (Algorithm 2): R = RN(T + inc), then the
    error-free sum of (V, R): V' + T' = V + R exactly (sum_3op when
    |V| >= |R|) and V' = RN(V + R); R from numpy's binary16 arithmetic."""
    V, T, inc = _update_inputs(40 + comp, O.FP16)
    inc = np.asarray(inc, np.float16).astype(np.float64)
    R = (T.astype(np.float16) + inc.astype(np.float16)).astype(np.float64)
    Vo, To = O.solution_update(comp, V, T, inc, O.FP16, O.FP16)
    ok = np.isfinite(R) & (np.abs(V + R) <= 65504.0)
    if comp == 3:
        ok &= np.abs(V) >= np.abs(R)
    assert ok.sum() > 100_000
    assert np.array_equal((Vo + To)[ok], (V + R)[ok])
    assert np.array_equal(Vo[ok], np.asarray(V + R, np.float16).astype(np.float64)[ok])
    # T dropped from R breaks the identity
    Vd, Td = O.solution_update(comp, V, np.zeros_like(T), inc, O.FP16, O.FP16)
    assert np.any((Vd + Td)[ok] != (V + R)[ok])
