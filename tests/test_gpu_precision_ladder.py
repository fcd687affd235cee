"""Precision ladder on the GPU path: every storage / arithmetic / update
variant of the 3D acoustic and the 2D elastic scheme, its error against the
binary64 oracle run of the same problem and its energy drift, plus the
Appendix B stencil promotion (binary64 stencil, half update), which exists in
the oracle only. Run with -s to print the table.

Assertions are the orderings the paper reports: compensation reduces the
error and the energy drift of half storage; sum_3op and sum_6op agree far
better than either agrees with the plain update; promoting the stencil alone
does not stop the plain update's drift; binary32 is far below all half
variants.
"""
import numpy as np
import pytest

import oracle as O
from paper_2310_00236_gb300 import inputs
from paper_2310_00236_gb300 import wave as W
from wave_helpers import PREC

pytestmark = pytest.mark.gpu
R = W.WAVE_BC_RIGID
VARIANTS = [("fp16", 0), ("fp16", 3), ("fp16", 6), ("bf16", 0), ("bf16", 3), ("bf16", 6),
            ("fp16_f32arith", 0), ("fp16_f32arith", 3), ("bf16_f32arith", 3), ("fp32", 0)]
# the paper's variants and the pair precision (not the paper's scheme)
LADDER = VARIANTS + [("fp16_pairs", 3)]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_precision_ladder_3d_acoustic():
    n, steps = 64, 400
    shape = (n, n, n)
    w = inputs.acoustic_3d_random(n=n, sigma_cells=2.0, ic_sigma_cells=3.0, smooth_dtype=np.float64)
    ref = O.acoustic_setup(shape, (1, 1, 1), w["h"], w["dt"], w["rho"], w["c"], O.FP64, 0, p0=w["p0"])
    _, E = ref.run(steps, energy=True)
    rows = {}
    for prec, comp in LADDER:
        code = PREC[prec][0]
        ctx = W.wave_create(shape, w["h"], w["rho"], w["c"], w["dt"], code, comp, bc=[R] * 6)
        try:
            W.wave_set_initial(ctx, W.WAVE_F_P, w["p0"])
            W.wave_step(ctx, 1)
            e0 = W.wave_energy(ctx)
            W.wave_step(ctx, steps - 1)
            e1 = W.wave_energy(ctx)
            p = W.wave_get_field(ctx, W.WAVE_F_P).reshape(ref.p.shape)
        finally:
            W.wave_destroy(ctx)
        rows[(prec, comp)] = (_rel(p, ref.p), (e1 - e0) / e0)
    # Appendix B: binary64 stencil with a binary16 update (oracle only)
    for comp in (0, 3):
        st = O.acoustic_setup(shape, (1, 1, 1), w["h"], w["dt"], w["rho"], w["c"], O.FP16, comp, p0=w["p0"],
                              stencil_fmt=O.FP64)
        _, Es = st.run(steps, energy=True)
        rows[("fp16+fp64 stencil", comp)] = (_rel(st.p, ref.p), (Es[-1] - Es[0]) / Es[0])
    print(f"\n3D acoustic {n}^3, {steps} steps, CFL 0.4; FP64 energy drift {(E[-1] - E[0]) / E[0]:.2e}")
    for k, (err, drift) in rows.items():
        print(f"  {k[0]:>20s} comp={k[1]}  rel L2 vs FP64 {err:.3e}  energy drift {drift:+.3e}")
    assert rows[("fp32", 0)][0] < 1e-4
    for s in ("fp16", "bf16"):
        assert abs(rows[(s, 3)][1]) < abs(rows[(s, 0)][1])
        assert _close(rows[(s, 3)], rows[(s, 6)], rows[(s, 0)])
    assert abs(rows[("fp16_f32arith", 3)][1]) < abs(rows[("fp16_f32arith", 0)][1])
    # reading the pair V + T (and binary32 multipliers) removes the stored
    # value's and the multipliers' rounding: under the 2e-3 bar, an order of
    # magnitude below the stored-value stencil
    assert rows[("fp16_pairs", 3)][0] < min(2e-3, 0.2 * rows[("fp16_f32arith", 3)][0])
    assert abs(rows[("fp16+fp64 stencil", 3)][1]) < abs(rows[("fp16+fp64 stencil", 0)][1])
    for k, (err, _) in rows.items():
        if k != ("fp32", 0):
            assert err > 10 * rows[("fp32", 0)][0]


def _close(a, b, plain):
    """3op and 6op agree better than either agrees with the plain update."""
    return abs(a[1] - b[1]) <= abs(a[1] - plain[1])


def test_precision_ladder_2d_elastic():
    n, steps = 192, 1200
    shape = (n, n)
    w = inputs.elastic_2d_layered(n=n, steps=steps)
    bc = (O.EBC_RIGID, O.EBC_RIGID, O.EBC_FREE, O.EBC_RIGID)
    P0 = 1e5
    z0 = float(w["rho"].max() * w["vp"].max())
    amp = 0.5 * P0 * w["h"] ** 2 / (w["dt"] * z0)
    idx = list(w["src_idx"])
    ref = O.elastic_setup(shape, bc, w["h"], w["dt"], w["rho"], w["vp"], w["vs"], O.FP64, 0, P0=P0)
    ref.src_index = idx[0] + n * idx[1]
    ref.src = O.elastic_scale_source(w["wavelet"] * amp, w["dt"], ref.Z0, P0, w["h"], O.FP64)
    _, E = ref.run(steps, energy=True)
    quiet = w["src_steps"] + 1
    names = ("vx", "vy", "sxx", "syy", "sxy")
    fids = (W.WAVE_F_VX, W.WAVE_F_VY, W.WAVE_F_SXX, W.WAVE_F_SYY, W.WAVE_F_SXY)
    refv = np.concatenate([ref.f[k].ravel() for k in names])
    rows = {}
    for prec, comp in LADDER:
        code = PREC[prec][0]
        ctx = W.wave_create(shape, w["h"], w["rho"], w["vp"], w["dt"], code, comp, vs=w["vs"],
                            bc=[1, 1, 2, 1, 0, 0], kind=W.WAVE_ELASTIC, field_scale=P0)
        try:
            W.wave_set_source(ctx, W.WAVE_F_VY, idx, w["wavelet"] * amp)
            W.wave_step(ctx, quiet)
            e0 = W.wave_energy(ctx)
            W.wave_step(ctx, steps - quiet)
            e1 = W.wave_energy(ctx)
            got = np.concatenate([W.wave_get_raw(ctx, f, 0).astype(np.float64).ravel() if prec == "fp32"
                                  else _raw_values(W.wave_get_raw(ctx, f, 0), prec) for f in fids])
        finally:
            W.wave_destroy(ctx)
        rows[(prec, comp)] = (_rel(got, refv), (e1 - e0) / e0)
    e_ref = (E[-1] - E[quiet - 1]) / E[quiet - 1]
    print(f"\n2D elastic {n}^2, {steps} steps (source off after step {quiet}); FP64 drift {e_ref:.2e}")
    for k, (err, drift) in rows.items():
        print(f"  {k[0]:>20s} comp={k[1]}  rel L2 vs FP64 {err:.3e}  energy drift {drift:+.3e}")
    assert rows[("fp32", 0)][0] < 1e-4
    for s in ("fp16", "bf16"):
        assert abs(rows[(s, 3)][1]) < abs(rows[(s, 0)][1])
        assert _close(rows[(s, 3)], rows[(s, 6)], rows[(s, 0)])
    # the pair precision reads V + T in its stencils (and binary32 multipliers)
    assert rows[("fp16_pairs", 3)][0] < 0.2 * rows[("fp16_f32arith", 3)][0]
    for k, (err, _) in rows.items():
        if k != ("fp32", 0):
            assert err > 10 * rows[("fp32", 0)][0]


def _raw_values(raw, prec):
    if prec.startswith("bf16"):
        import torch
        return torch.from_numpy(raw.view(np.int16).copy()).view(torch.bfloat16).to(torch.float64).numpy().ravel()
    return raw.view(np.float16).astype(np.float64).ravel()
