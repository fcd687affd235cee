"""Pins of the oracle's pair reading (pair_stencil: every stencil tap reads
RN32(V + T), the stored value plus its carried compensation; binary16 storage,
binary32 arithmetic). Beside its accuracy against binary64
(test_oracle_accuracy_split.py), two properties fix what the taps read:

* the taps depend on V and T only through their sum: exchanging the stored
  p and its compensation t_p leaves the new velocities of a step unchanged
  (RN32(V + T) = RN32(T + V)), while the stored-value scheme, whose taps read
  V, changes them;
* with every T zero the taps are the stored values, so the first velocity
  half step equals the stored-value scheme's.

A tap that read V alone, dropped T, subtracted it, or read T twice fails one
of them.
"""
import numpy as np
import pytest

import oracle as O


def _state(pairs, shape=(24, 20), seed=3):
    rng = np.random.default_rng(seed)
    nd = len(shape)
    h, dt = 10.0, 0.4 * 10.0 / 4500.0
    c = 1500.0 + 3000.0 * rng.random(shape[::-1])
    rho = 1000.0 + 1600.0 * rng.random(shape[::-1])
    st = O.acoustic_setup(shape, (O.BC_RIGID,) * nd, h, dt, rho, c, O.FP16, 3, arith_fmt=O.FP32,
                          pair_stencil=pairs, coef_fmt=O.FP32 if pairs else None)
    # binary16 V and a T of about one unit in the last place of V
    st.p = O.round_to(rng.standard_normal(st.shape), O.FP16)
    st.tp = O.round_to(st.p * rng.uniform(-1e-3, 1e-3, st.shape), O.FP16)
    for ax in range(nd):
        st.v[ax] = O.round_to(0.3 * rng.standard_normal(st.shape), O.FP16)
    st.apply_walls()
    return st


@pytest.mark.parametrize("pairs", [True, False])
def test_taps_read_the_sum_of_v_and_t(oracle_lib, pairs):
    st = _state(pairs)
    sw = st.copy()
    sw.p, sw.tp = st.tp.copy(), st.p.copy()
    assert np.any(st.tp != 0)
    st.run(1)
    sw.run(1)
    same = all(np.array_equal(st.v[a], sw.v[a]) and np.array_equal(st.tv[a], sw.tv[a]) for a in range(2))
    # the pair taps see the same sums; the stored-value taps see other values
    assert same == pairs


def test_zero_compensation_reduces_to_the_stored_value_scheme(oracle_lib):
    pr = _state(True)
    sv = _state(False)
    pr.tp[:] = 0.0
    sv.tp[:] = 0.0
    # the same multipliers on both sides (the pair reading keeps them in binary32)
    sv.a = [x.copy() for x in pr.a]
    sv.b = pr.b.copy()
    pr.run(1)
    sv.run(1)
    for a in range(2):
        assert np.array_equal(pr.v[a], sv.v[a]) and np.array_equal(pr.tv[a], sv.tv[a])
    assert np.any(pr.v[0] != 0)
