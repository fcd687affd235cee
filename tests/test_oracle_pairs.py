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
of them. The same pins hold the elastic reading (the stresses' taps in the
velocity half step), with its accuracy against binary64 on the layered
free-surface model.
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


# ------------------------------------------------------------------ elastic
def _elastic(pairs, fmt=O.FP16, comp=3, n=48, seed=5):
    """Layered medium, free top, rigid sides; random binary16 fields with a
    compensation of about one unit in the last place."""
    from paper_2310_00236_gb300 import inputs
    w = inputs.elastic_2d_layered(n=n, steps=10)
    bc = (O.EBC_RIGID, O.EBC_RIGID, O.EBC_FREE, O.EBC_RIGID)
    kw = dict(arith_fmt=O.FP32, pair_stencil=True, coef_fmt=O.FP32) if pairs else \
        (dict(arith_fmt=O.FP32) if fmt == O.FP16 else {})
    st = O.elastic_setup((n, n), bc, w["h"], w["dt"], w["rho"], w["vp"], w["vs"], fmt, comp, P0=1e5, **kw)
    rng = np.random.default_rng(seed)
    for k in O.ELASTIC_FIELDS:
        st.f[k] = O.round_to(rng.standard_normal(st.shape), fmt)
        if comp:
            st.t[k] = O.round_to(st.f[k] * rng.uniform(-1e-3, 1e-3, st.shape), fmt)
    st.apply_walls()
    st.t["syy"][0, :] = 0.0  # held with syy on the free-surface row
    return st, w


@pytest.mark.parametrize("pairs", [True, False])
def test_elastic_taps_read_the_sum_of_v_and_t(oracle_lib, pairs):
    """Exchanging every stress with its compensation leaves the new
    velocities unchanged for the pair taps only."""
    st, _ = _elastic(pairs)
    sw, _ = _elastic(pairs)
    for k in ("sxx", "syy", "sxy"):
        sw.f[k], sw.t[k] = st.t[k].copy(), st.f[k].copy()
    st.run(1)
    sw.run(1)
    same = all(np.array_equal(st.f[k], sw.f[k]) and np.array_equal(st.t[k], sw.t[k]) for k in ("vx", "vy"))
    assert same == pairs


def test_elastic_zero_compensation_reduces_to_the_stored_value_scheme(oracle_lib):
    pr, _ = _elastic(True)
    sv, _ = _elastic(False)
    for k in O.ELASTIC_FIELDS:
        pr.t[k][:] = 0.0
        sv.t[k][:] = 0.0
        sv.f[k] = pr.f[k].copy()
    sv.coef = {k: v.copy() for k, v in pr.coef.items()}
    pr.run(1)
    sv.run(1)
    for k in ("vx", "vy"):
        assert np.array_equal(pr.f[k], sv.f[k]) and np.array_equal(pr.t[k], sv.t[k])


def test_elastic_pairs_accuracy_against_binary64(oracle_lib):
    """A Ricker force under the free surface of the layered model, 96^2, 600
    steps: the pair reading within 1e-3 of the binary64 run and at least five
    times closer than fp16 + sum_3op."""
    from paper_2310_00236_gb300 import inputs
    n, steps = 96, 600
    w = inputs.elastic_2d_layered(n=n, steps=steps)
    bc = (O.EBC_RIGID, O.EBC_RIGID, O.EBC_FREE, O.EBC_RIGID)

    def run(fmt, comp, **kw):
        st = O.elastic_setup((n, n), bc, w["h"], w["dt"], w["rho"], w["vp"], w["vs"], fmt, comp, P0=1e5, **kw)
        amp = 0.5 * 1e5 * w["h"] ** 2 / (w["dt"] * st.Z0)
        st.src = O.elastic_scale_source(w["wavelet"] * amp, w["dt"], st.Z0, 1e5, w["h"], kw.get("arith_fmt", fmt))
        st.src_index = int(np.ravel_multi_index((10, n // 2), st.shape))
        st.run(steps)
        return st.f["vy"]

    ref = run(O.FP64, 0)
    rel = lambda a: float(np.linalg.norm(a - ref) / np.linalg.norm(ref))
    k3 = rel(run(O.FP16, 3))
    pairs = rel(run(O.FP16, 3, arith_fmt=O.FP32, pair_stencil=True, coef_fmt=O.FP32))
    assert pairs < 1e-3 and pairs * 5 < k3, (pairs, k3)
