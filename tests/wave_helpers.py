"""Shared helpers for the parity tests: run the same seeded inputs through the
CUDA path (C ABI via the ctypes binding) and through the CPU oracle, and
compare stored bits."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2310_00236_gb300 import wave as W

# precision name -> (binding code, oracle storage format, oracle arithmetic format)
PREC = {
    "fp16": (W.WAVE_FP16, O.FP16, O.FP16),
    "bf16": (W.WAVE_BF16, O.BF16, O.BF16),
    "fp32": (W.WAVE_FP32, O.FP32, O.FP32),
    "fp16_f32arith": (W.WAVE_FP16_F32ARITH, O.FP16, O.FP32),
    "bf16_f32arith": (W.WAVE_BF16_F32ARITH, O.BF16, O.FP32),
    # stencils read RN32(V + T), multipliers in binary32: the oracle's
    # pair_stencil and coef_fmt readings
    "fp16_pairs": (W.WAVE_FP16_PAIRS, O.FP16, O.FP32),
}
PAIRS = {"fp16_pairs"}


def to_bits(values: np.ndarray, fmt: int) -> np.ndarray:
    """Exact encoding of oracle values (representable in fmt) as storage bits."""
    if fmt == O.FP16:
        return values.astype(np.float16).view(np.uint16)
    if fmt == O.FP32:
        return values.astype(np.float32).view(np.uint32)
    if fmt == O.BF16:
        import torch
        t = torch.from_numpy(values.astype(np.float32)).to(torch.bfloat16)
        return t.view(torch.int16).numpy().view(np.uint16)
    raise ValueError(fmt)


def gpu_bits(raw: np.ndarray) -> np.ndarray:
    return raw.view(np.uint32) if raw.dtype == np.float32 else raw


def acoustic_pair(shape, bc, prec, comp, h, dt, rho, c, p0=None, v0=None, P0=1.0, src=None,
                  rec=None, kernel=0, zchunk=0, stream=None):
    """Create matching GPU context and oracle state. src = (idx, wavelet);
    rec = (field, list of idx). Returns (ctx, oracle_state)."""
    code, sfmt, afmt = PREC[prec]
    nd = len(shape)
    bcw = []
    for ax in range(3):
        b = bc[ax] if ax < nd else W.WAVE_BC_PERIODIC
        bcw += [b, b]
    ctx = W.wave_create(shape, h, rho, c, dt, code, comp, bc=bcw, field_scale=P0, kernel=kernel,
                        zchunk=zchunk, stream=stream)
    # the pair precision: stencils read RN32(V + T), multipliers in binary32
    pairs = prec in PAIRS
    st = O.acoustic_setup(shape, bc, h, dt, rho, c, sfmt, comp, P0=P0, arith_fmt=afmt,
                          p0=p0, v0=v0, pair_stencil=pairs, coef_fmt=O.FP32 if pairs else None)
    if p0 is not None:
        W.wave_set_initial(ctx, W.WAVE_F_P, p0)
    if v0 is not None:
        for ax, vv in enumerate(v0):
            if vv is not None:
                W.wave_set_initial(ctx, W.WAVE_F_VX + ax, vv)
    if src is not None:
        idx, wav = src
        W.wave_set_source(ctx, W.WAVE_F_P, idx, wav)
        st.src_index = int(np.ravel_multi_index(tuple(idx[::-1]), st.shape))
        st.src = O.scale_source(wav, st.Z0, P0, h, nd, afmt)
    return ctx, st


def compare_acoustic(ctx, st, prec, comp):
    """Bit-exact comparison of every field and compensation. Returns list of
    mismatch descriptions (empty when identical)."""
    _, sfmt, _ = PREC[prec]
    nd = ctx.ndim
    bad = []
    fields = [("p", W.WAVE_F_P, st.p, st.tp)] + [
        ("v" + "xyz"[a], W.WAVE_F_VX + a, st.v[a], st.tv[a]) for a in range(nd)]
    for name, fid, val, comp_arr in fields:
        for is_comp, ref in ((0, val), (1, comp_arr)):
            if is_comp and not comp:
                continue
            if not np.all(np.isfinite(ref)):
                bad.append(f"{name}: oracle state is not finite (test inputs out of range)")
                continue
            g = gpu_bits(W.wave_get_raw(ctx, fid, is_comp))
            r = to_bits(ref, sfmt)
            if not np.array_equal(g, r):
                n = int(np.count_nonzero(g != r))
                first = np.argwhere(g != r)[0]
                bad.append(f"{name}{'(comp)' if is_comp else ''}: {n} mismatches, first at "
                           f"{tuple(first)} gpu={g[tuple(first)]:#x} oracle={r[tuple(first)]:#x}")
    return bad
