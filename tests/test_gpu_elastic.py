"""GPU parity of the 2D elastic path against the CPU oracle (bit-exact).

Every stored value of the five fields (vx, vy, sxx, syy, sxy) and their
compensations equals the oracle's op-by-op emulation, for every precision and
update variant, with periodic, rigid and free faces, layered media, a v_y
source, receivers and the fused energy. Full size: the 1024^2 three-layer
workload (free top, rigid sides), sampled points checked against oracle runs
over light-cone sub-boxes with the full-grid multipliers.
"""
import numpy as np
import pytest

import oracle as O
from paper_2310_00236_gb300 import wave as W
from wave_helpers import PAIRS, PREC, gpu_bits, to_bits

pytestmark = pytest.mark.gpu
PER, RIG, FREE = W.WAVE_BC_PERIODIC, W.WAVE_BC_RIGID, W.WAVE_BC_FREE
FIELDS = [("vx", W.WAVE_F_VX), ("vy", W.WAVE_F_VY), ("sxx", W.WAVE_F_SXX),
          ("syy", W.WAVE_F_SYY), ("sxy", W.WAVE_F_SXY)]


def layered(shape, seed=0, smooth=True):
    """Three horizontal layers (Vp 2000/3000/4000, Vs = Vp/1.73, rho
    2000/2300/2600) with a small seeded perturbation."""
    nx, ny = shape
    y = np.arange(ny)
    vp = np.where(y < ny // 3, 2000.0, np.where(y < 2 * ny // 3, 3000.0, 4000.0))
    rho = np.where(y < ny // 3, 2000.0, np.where(y < 2 * ny // 3, 2300.0, 2600.0))
    vp = np.repeat(vp[:, None], nx, 1)
    rho = np.repeat(rho[:, None], nx, 1)
    if smooth:
        rng = np.random.default_rng(seed)
        vp = vp * (1.0 + 0.02 * rng.uniform(-1, 1, vp.shape))
        rho = rho * (1.0 + 0.02 * rng.uniform(-1, 1, rho.shape))
    return rho, np.minimum(vp, 4000.0), np.minimum(vp, 4000.0) / 1.73


def elastic_pair(shape, bc, prec, comp, h, dt, rho, vp, vs, init, P0, src=None, kernel=0):
    code, sfmt, afmt = PREC[prec]
    ctx = W.wave_create(shape, h, rho, vp, dt, code, comp, vs=vs, bc=list(bc) + [0, 0],
                        kind=W.WAVE_ELASTIC, field_scale=P0, kernel=kernel)
    # the pair precision: stencil taps RN32(V + T), multipliers in binary32
    pairs = prec in PAIRS
    st = O.elastic_setup(shape, bc, h, dt, rho, vp, vs, sfmt, comp, P0=P0, arith_fmt=afmt,
                         init=init, pair_stencil=pairs, coef_fmt=O.FP32 if pairs else None)
    for name, fid in FIELDS:
        if name in init:
            W.wave_set_initial(ctx, fid, init[name])
    if src is not None:
        idx, wav = src
        W.wave_set_source(ctx, W.WAVE_F_VY, idx, wav)
        st.src_index = idx[0] + shape[0] * idx[1]
        st.src = O.elastic_scale_source(wav, dt, st.Z0, P0, h, afmt)
    return ctx, st


def compare(ctx, st, prec, comp):
    _, sfmt, _ = PREC[prec]
    bad = []
    for name, fid in FIELDS:
        for is_comp, ref in ((0, st.f[name]), (1, st.t[name])):
            if is_comp and not comp:
                continue
            if not np.all(np.isfinite(ref)):
                bad.append(f"{name}: oracle not finite")
                continue
            g = gpu_bits(W.wave_get_raw(ctx, fid, is_comp))
            r = to_bits(ref, sfmt)
            if not np.array_equal(g, r):
                first = tuple(np.argwhere(g != r)[0])
                bad.append(f"{name}{'(t)' if is_comp else ''}: {int(np.count_nonzero(g != r))} "
                           f"mismatches, first {first} gpu {g[first]:#x} oracle {r[first]:#x}")
    return bad


def _init(shape, seed, P0):
    rng = np.random.default_rng(seed)
    nx, ny = shape
    x = np.arange(nx)
    y = np.arange(ny)
    X, Y = np.meshgrid(x, y)
    g = np.exp(-((X - nx / 2) ** 2 + (Y - ny / 3) ** 2) / 20.0) * P0
    return {"sxx": g + 0.05 * P0 * rng.standard_normal(g.shape),
            "syy": g, "sxy": 0.1 * P0 * rng.standard_normal(g.shape),
            "vx": 0.02 * P0 / 1.04e7 * rng.standard_normal(g.shape)}


def _run(shape, bc, prec, comp, steps, src=False, energy=False, seed=0, kernel=0):
    h = 3.0
    rho, vp, vs = layered(shape, seed)
    dt = 0.5 * h / 4000.0
    P0 = 1e5
    s = None
    if src:
        z0 = float(rho.max() * vp.max())
        wav = np.sin(np.arange(steps) * 0.3) * 0.5 * P0 * h * h / (dt * z0)
        s = ([shape[0] // 2, min(10, shape[1] - 1)], wav)
    ctx, st = elastic_pair(shape, bc, prec, comp, h, dt, rho, vp, vs, _init(shape, seed, P0), P0, s,
                           kernel=kernel)
    try:
        W.wave_step(ctx, steps)
        _, E = st.run(steps, energy=energy)
        bad = compare(ctx, st, prec, comp)
        if energy:
            e_gpu = W.wave_energy(ctx)
            e_orc = E[-1] * 0.5 * h * P0 * P0 * dt / st.Z0
            if not abs(e_gpu - e_orc) <= 1e-9 * abs(e_orc):
                bad.append(f"energy {e_gpu} vs {e_orc}")
    finally:
        W.wave_destroy(ctx)
    assert not bad, bad


VARIANTS = [("fp16", 0), ("fp16", 3), ("fp16", 6), ("bf16", 3), ("bf16", 6), ("fp32", 0),
            ("fp32", 3), ("fp16_f32arith", 3), ("bf16_f32arith", 0), ("fp16_pairs", 3)]
BCS = [(RIG, RIG, FREE, RIG), (PER, PER, FREE, RIG), (PER, PER, PER, PER), (RIG, RIG, RIG, RIG)]


# kernel 0: row strips (the default); kernel 1: one thread per point
@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("prec,comp", VARIANTS)
def test_elastic_bit_exact_free_top_rigid_sides(prec, comp, kernel):
    _run((37, 29), BCS[0], prec, comp, 25, src=True, energy=True, kernel=kernel)


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("bc", BCS)
def test_elastic_bit_exact_all_boundaries(bc, kernel):
    _run((64, 48), bc, "fp16", 6, 30, src=True, energy=True, kernel=kernel)
    _run((8, 8), bc, "fp16", 3, 20, kernel=kernel)


@pytest.mark.parametrize("shape", [(257, 40), (300, 23), (513, 17), (9, 70)])
@pytest.mark.parametrize("bc", [BCS[0], BCS[2]])
def test_elastic_strips_ragged(shape, bc):
    # strips cut by the grid's x extent (ragged last vector, lanes past the
    # grid), periodic x wrapping across strip boundaries, row chunks cut by ny
    _run(shape, bc, "fp16", 3, 12, src=True, energy=True)
    _run(shape, bc, "fp32", 0, 12, energy=True)


def test_elastic_receivers():
    import torch
    shape = (40, 32)
    h = 3.0
    rho, vp, vs = layered(shape, 1)
    dt = 0.5 * h / 4000.0
    P0 = 1e5
    steps = 40
    z0 = float(rho.max() * vp.max())
    wav = np.sin(np.arange(steps) * 0.2) * 0.5 * P0 * h * h / (dt * z0)
    ctx, st = elastic_pair(shape, BCS[0], "fp16", 6, h, dt, rho, vp, vs, {}, P0,
                           ([20, 10], wav))
    recs = [(5, 10), (30, 10), (39, 31)]
    try:
        tr = torch.zeros(steps * len(recs), dtype=torch.float32, device="cuda")
        W.wave_set_receivers(ctx, W.WAVE_F_VY, recs, tr, steps)
        W.wave_step(ctx, steps)
        traces, _ = st.run(steps, rec_field=2, rec_index=[i + shape[0] * j for i, j in recs])
        got = tr.cpu().numpy().reshape(steps, len(recs)).astype(np.float64)
        assert np.array_equal(got, traces)
        assert np.any(got != 0)
    finally:
        W.wave_destroy(ctx)


def test_elastic_coefficients_bit_exact():
    shape = (33, 27)
    rho, vp, vs = layered(shape, 2)
    for prec in ("fp16", "bf16", "fp32"):
        code, sfmt, _ = PREC[prec]
        ctx = W.wave_create(shape, 3.0, rho, vp, 3.75e-4, code, 6, vs=vs, bc=list(BCS[0]) + [0, 0],
                            kind=W.WAVE_ELASTIC)
        cfg = O.elastic_cfg(shape, BCS[0], sfmt, 6)
        coef, z0, ok = O.elastic_coefficients(cfg, 3.0, 3.75e-4, rho, vp, vs)
        assert ok
        try:
            for w, name in enumerate(("bx", "by", "l2m", "lam", "mu")):
                g, gz = W.wave_get_coefficient(ctx, w)
                assert gz == z0
                assert np.array_equal(g, coef[name]), name
        finally:
            W.wave_destroy(ctx)


def test_elastic_full_size_1024_sampled_bit_exact():
    """1024^2 three-layer model (h = 3 m, dt = 0.5 h / 4000), free top, rigid
    sides, fp16 + sum_6op, random stresses everywhere, 4 steps."""
    n = 1024
    shape = (n, n)
    h = 3.0
    rho, vp, vs = layered(shape, 0, smooth=False)
    dt = 0.5 * h / 4000.0
    P0 = 1e5
    steps = 4
    prec, comp = "fp16", 6
    code, sfmt, afmt = PREC[prec]
    rng = np.random.default_rng(4)
    init = {k: P0 * rng.standard_normal(shape[::-1]) for k in ("sxx", "syy", "sxy")}
    init["vy"] = P0 / 1.04e7 * rng.standard_normal(shape[::-1])
    ctx = W.wave_create(shape, h, rho, vp, dt, code, comp, vs=vs, bc=list(BCS[0]) + [0, 0],
                        kind=W.WAVE_ELASTIC, field_scale=P0)
    try:
        for name, fid in FIELDS:
            if name in init:
                W.wave_set_initial(ctx, fid, init[name])
        W.wave_step(ctx, steps)
        got = {name: gpu_bits(W.wave_get_raw(ctx, fid, 0)) for name, fid in FIELDS}
        got.update({name + "_t": gpu_bits(W.wave_get_raw(ctx, fid, 1)) for name, fid in FIELDS})
    finally:
        W.wave_destroy(ctx)
    full = O.elastic_setup(shape, BCS[0], h, dt, rho, vp, vs, sfmt, comp, P0=P0, arith_fmt=afmt,
                           init=init)
    M = 4 * steps + 4
    pts = [(0, 0), (n - 1, n - 1), (n // 2, 0), (0, n // 2), (n - 1, 3), (5, n - 1), (n // 2, n // 2),
           (n // 3, n // 3 + 1), (2 * n // 3, 2 * n // 3)]
    pts += [tuple(int(x) for x in rng.integers(0, n, 2)) for _ in range(16)]
    bad = []
    for (i, j) in pts:
        lo = [max(0, i - M), max(0, j - M)]
        hi = [min(n, i + M + 1), min(n, j + M + 1)]
        # real faces keep their kind; cut faces read zero (their influence
        # stays outside the checked point's domain of dependence)
        Z = O.EBC_ZERO
        bc = (RIG if lo[0] == 0 else Z, RIG if hi[0] == n else Z,
              FREE if lo[1] == 0 else Z, RIG if hi[1] == n else Z)
        sub = (hi[0] - lo[0], hi[1] - lo[1])
        cfg = O.elastic_cfg(sub, bc, sfmt, comp, afmt)
        st = O.ElasticState(cfg)
        sl = (slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        for k in st.coef:
            st.coef[k] = np.ascontiguousarray(full.coef[k][sl])
        for k in st.f:
            st.f[k] = np.ascontiguousarray(full.f[k][sl])
        st.run(steps)
        li, lj = i - lo[0], j - lo[1]
        for name, _ in FIELDS:
            for suffix, arr in (("", st.f[name]), ("_t", st.t[name])):
                g = got[name + suffix][j, i]
                r = to_bits(np.array([arr[lj, li]]), sfmt)[0]
                if g != r:
                    bad.append(f"{name}{suffix} at {(i, j)}: gpu {g:#x} oracle {r:#x}")
    assert not bad, bad[:10]


def test_elastic_graph_replay_on_side_stream_bit_exact():
    """Plain elastic stepping on a created stream replays captured step graphs
    (the step index of the source lives in device memory): oracle bits across
    calls, with the source active."""
    import torch
    shape = (70, 44)
    h = 3.0
    rho, vp, vs = layered(shape, 3)
    dt = 0.5 * h / 4000.0
    P0 = 1e5
    steps = [70, 40, 3]
    n = sum(steps)
    z0 = float(rho.max() * vp.max())
    wav = np.sin(np.arange(n) * 0.2) * 0.5 * P0 * h * h / (dt * z0)
    code, sfmt, afmt = PREC["fp16"]
    stream = torch.cuda.Stream()
    ctx = W.wave_create(shape, h, rho, vp, dt, code, 6, vs=vs, bc=list(BCS[0]) + [0, 0],
                        kind=W.WAVE_ELASTIC, field_scale=P0, stream=stream.cuda_stream)
    st = O.elastic_setup(shape, BCS[0], h, dt, rho, vp, vs, sfmt, 6, P0=P0, arith_fmt=afmt,
                         init=_init(shape, 3, P0))
    try:
        for name, fid in FIELDS:
            W.wave_set_initial(ctx, fid, _init(shape, 3, P0)[name]) if name in ("sxx", "syy", "sxy", "vx") else None
        W.wave_set_source(ctx, W.WAVE_F_VY, [35, 10], wav)
        st.src_index = 35 + shape[0] * 10
        st.src = O.elastic_scale_source(wav, dt, st.Z0, P0, h, afmt)
        for m in steps:
            W.wave_step(ctx, m)
        st.run(n)
        bad = compare(ctx, st, "fp16", 6)
    finally:
        W.wave_destroy(ctx)
    assert not bad, bad
