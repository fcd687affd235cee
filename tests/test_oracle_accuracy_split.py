"""The error split of the half-precision scheme (Section 5, "Operator" and
"Range"), checked at reduced size with the CPU oracle (tests/accuracy_split.py
prints the full-size tables).

* the 2D acoustic 256^2 problem (rho = c = 1, CFL 0.5): the multipliers a = b = 1/2 are exact in
  binary16, so their rounding costs nothing; rounding the weight 1/24 alone
  costs about a third of the method's error; half storage with the
  compensation carried and every other operation and coefficient in binary64
  gives nearly all of it. So no choice of coefficient precision brings
  fp16 + sum_3op under 2e-3 there, while a stencil that reads the stored
  pair V + T in binary32 (not the paper's scheme) does.
* W0 regime (CFL 0.0125): a = b = 0.0125 are not binary16 numbers; their
  rounding alone is the largest single part of the error.
"""
import numpy as np
import pytest

import accuracy_split as A
import oracle as O


def _err(case, ref, **kw):
    out, _ = A.run(case, **kw)
    return float(np.linalg.norm(out - ref) / np.linalg.norm(ref))


def test_split_acoustic2d_256(oracle_lib):
    case = A.acoustic2d_256(small=True)
    ref, _ = A.run(case, store_fmt=O.FP64, comp=0)
    method = _err(case, ref, store_fmt=O.FP16, comp=3)
    coef = _err(case, ref, store_fmt=O.FP64, comp=0, coef_fmt=O.FP16)
    c2 = _err(case, ref, store_fmt=O.FP64, comp=0, c2_fmt=O.FP16)
    storage = _err(case, ref, store_fmt=O.FP16, comp=3, arith_fmt=O.FP64, stencil_fmt=O.FP64,
                   coef_fmt=O.FP64)
    pairs = _err(case, ref, store_fmt=O.FP16, comp=3, arith_fmt=O.FP32, pair_stencil=True,
                 coef_fmt=O.FP32)
    assert method > 2e-3, method
    assert coef == 0.0
    assert 0.15 * method < c2 < 0.45 * method, (c2, method)
    assert abs(storage - method) < 0.1 * method, (storage, method)
    assert pairs < 2e-3 and pairs < 0.1 * method, (pairs, method)


def test_split_w0_regime(oracle_lib):
    n, steps = 80, 6000
    case = dict(A.w0(small=True))
    h, dt = case["h"], case["dt"]
    wav = A.inputs.ricker_table(steps, dt, 5.0)
    case.update(shape=(n, n), rho=np.ones((n, n)), c=np.ones((n, n)), steps=steps,
                src=(n // 3, n // 3, wav * 0.5 * h), rec=(2 * n // 3, 2 * n // 3))
    ref, _ = A.run(case, store_fmt=O.FP64, comp=0)
    method = _err(case, ref, store_fmt=O.FP16, comp=3)
    coef = _err(case, ref, store_fmt=O.FP64, comp=0, coef_fmt=O.FP16)
    storage = _err(case, ref, store_fmt=O.FP16, comp=3, arith_fmt=O.FP64, stencil_fmt=O.FP64,
                   coef_fmt=O.FP64)
    # 0.0125 rounds to 0.012496948..., a -2.4e-4 change of each multiplier
    assert A.O.round_to(np.array([0.0125]), O.FP16)[0] != 0.0125
    assert coef > storage and coef > 0.5 * method, (coef, storage, method)
