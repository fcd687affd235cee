"""GPU parity of the 3D streaming kernels (two-kernel and one-pass) against the CPU oracle.

Small grids: bit-exact on every stored value, with x tiles that end inside
the grid, partial y tiles, several z chunks, both boundary kinds, a source and
the fused energy. Full size: the 512^3 benchmark workload in the launch
configuration the benchmark uses, checked bit for bit at sampled points; each
sample's expected value comes from an oracle run on a sub-box around it that
contains the point's whole domain of dependence (radius 4 per step + 4) and
carries the full-grid coefficients.
"""
import numpy as np
import pytest

import oracle as O
from paper_2310_00236_gb300 import inputs
from paper_2310_00236_gb300 import wave as W
from wave_helpers import PAIRS, PREC, acoustic_pair, compare_acoustic, gpu_bits, to_bits

pytestmark = pytest.mark.gpu
R, P = O.BC_RIGID, O.BC_PERIODIC

VARIANTS = [("fp16", 0), ("fp16", 3), ("fp16", 6), ("bf16", 3), ("bf16", 0), ("fp32", 0),
            ("fp32", 3), ("fp16_f32arith", 3), ("fp16_f32arith", 0), ("bf16_f32arith", 3),
            ("fp16_pairs", 3)]


def _media(shape, seed):
    c = inputs.smooth_random_field(shape, seed, 3.0, 1500.0, 4500.0)
    rho = inputs.smooth_random_field(shape, seed + 1, 3.0, 1000.0, 2600.0)
    return rho, c


def _run(shape, bc, prec, comp, steps, zchunk, src=False, energy=False, seed=0, kernel=2):
    """kernel 2 = the two-kernel streaming step."""
    h = 10.0
    rho, c = _media(shape, seed)
    dt = 0.4 * h / 4500.0 / np.sqrt(1.5)
    p0 = inputs.gaussian(shape, h, 3.0 * h)
    rng = np.random.default_rng(seed)
    v0 = [1e-4 * rng.standard_normal(p0.shape) for _ in range(3)]
    s = None
    if src:
        z0 = float(np.max(rho) * np.max(c))
        wav = inputs.ricker_table(steps, dt, 40.0) * 0.5 * h * h / z0
        s = ([shape[0] // 2 + 3, shape[1] // 3, shape[2] // 2], wav)
    ctx, st = acoustic_pair(shape, bc, prec, comp, h, dt, rho, c, p0=p0, v0=v0, src=s,
                            zchunk=zchunk, kernel=kernel)
    try:
        W.wave_step(ctx, steps)
        _, E = st.run(steps, energy=energy)
        bad = compare_acoustic(ctx, st, prec, comp)
        if energy:
            e_gpu = W.wave_energy(ctx)
            e_orc = E[-1] * O.energy_factor(h, dt, 1.0, st.Z0, 3)
            if not abs(e_gpu - e_orc) <= 2e-6 * abs(e_orc):
                bad.append(f"energy {e_gpu} vs oracle {e_orc}")
    finally:
        W.wave_destroy(ctx)
    assert not bad, bad


@pytest.mark.parametrize("prec,comp", VARIANTS)
def test_stream_ragged_tiles_rigid(prec, comp):
    nx = 72 if prec != "fp32" else 36
    _run((nx, 37, 29), (R, R, R), prec, comp, 6, zchunk=8, energy=True)


@pytest.mark.parametrize("prec,comp", [("fp16", 3), ("bf16", 6), ("fp32", 0), ("fp16_f32arith", 3),
                                       ("fp16_pairs", 3)])
def test_stream_periodic_and_mixed_with_source(prec, comp):
    nx = 128 if prec != "fp32" else 64
    _run((nx, 20, 17), (P, P, P), prec, comp, 7, zchunk=5, src=True)
    _run((nx, 33, 12), (R, P, R), prec, comp, 5, zchunk=64, src=True, energy=True)
    _run((nx, 16, 16), (P, R, P), prec, comp, 5, zchunk=3)


def test_stream_minimum_sizes():
    _run((8, 8, 8), (R, R, R), "fp16", 3, 9, zchunk=2, energy=True)
    _run((8, 9, 8), (P, R, P), "fp16_pairs", 3, 9, zchunk=1, energy=True)
    _run((8, 9, 8), (P, R, P), "fp16", 6, 9, zchunk=1)
    _run((12, 8, 9), (R, P, R), "fp32", 3, 9, zchunk=4, energy=True)


# -------------------------------------------------------------- full size
def _subbox_expect(w, st_full, prec, comp, steps, points):
    """Oracle values at `points` after `steps` steps, each from a sub-box run."""
    code, sfmt, afmt = PREC[prec]
    n = w["shape"][0]
    M = 4 * steps + 4
    out = []
    for (i, j, k) in points:
        lo = [max(0, c - M) for c in (i, j, k)]
        hi = [min(n, c + M + 1) for c in (i, j, k)]
        sl = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        shape = (hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2])
        cfg = O.acoustic_cfg(shape, (R, R, R), sfmt, comp, afmt, pair_stencil=prec in PAIRS)
        st = O.AcousticState(cfg)
        st.a = [np.ascontiguousarray(st_full["a"][ax][sl]) for ax in range(3)]
        st.b = np.ascontiguousarray(st_full["b"][sl])
        st.p = np.ascontiguousarray(st_full["p"][sl])
        for ax in range(3):
            st.v[ax] = np.ascontiguousarray(st_full["v"][ax][sl])
        st.apply_walls()
        st.run(steps)
        loc = (k - lo[2], j - lo[1], i - lo[0])
        vals = {"p": st.p[loc], "tp": st.tp[loc]}
        for ax in range(3):
            vals["v%d" % ax] = st.v[ax][loc]
            vals["tv%d" % ax] = st.tv[ax][loc]
        out.append(vals)
    return out


@pytest.mark.parametrize("prec,comp,kernel", [("fp16", 3, 0), ("fp32", 0, 0), ("fp16", 3, 3), ("fp16_pairs", 3, 0),
                                              ("fp16_pairs", 3, 2)])
def test_full_size_512_sampled_bit_exact(prec, comp, kernel):
    """The benchmark workload's grid and media (512^3, smooth random velocity,
    rho = 1000, p = 0 walls, CFL 0.4) in the benchmark's launch configuration,
    3 steps, sampled at corners, faces, edges, the centre and random interior
    points. Random pressure and velocities everywhere (on top of the Gaussian)
    so that every sample exercises the arithmetic."""
    steps = 3
    w = inputs.acoustic_3d_random(n=512)
    rng = np.random.default_rng(5)
    w["p0"] += 0.3 * rng.standard_normal(w["p0"].shape)
    z0 = 1000.0 * 4500.0
    v0 = [0.3 / z0 * rng.standard_normal(w["p0"].shape) for _ in range(3)]
    code, sfmt, afmt = PREC[prec]
    ctx = W.wave_create(w["shape"], w["h"], w["rho"], w["c"], w["dt"], code, comp,
                        bc=[W.WAVE_BC_RIGID] * 6, field_scale=w["P0"], kernel=kernel)
    try:
        W.wave_set_initial(ctx, W.WAVE_F_P, w["p0"])
        for ax in range(3):
            W.wave_set_initial(ctx, W.WAVE_F_VX + ax, v0[ax])
        W.wave_step(ctx, steps)
        got = {"p": gpu_bits(W.wave_get_raw(ctx, W.WAVE_F_P, 0))}
        if comp:
            got["tp"] = gpu_bits(W.wave_get_raw(ctx, W.WAVE_F_P, 1))
        for ax in range(3):
            got["v%d" % ax] = gpu_bits(W.wave_get_raw(ctx, W.WAVE_F_VX + ax, 0))
            if comp:
                got["tv%d" % ax] = gpu_bits(W.wave_get_raw(ctx, W.WAVE_F_VX + ax, 1))
    finally:
        W.wave_destroy(ctx)
    # full-grid coefficients (binary32 for the pair precision) and scaled
    # initial pressure from the oracle
    cfg = O.acoustic_cfg(w["shape"], (R, R, R), O.FP32 if prec in PAIRS else sfmt, comp, afmt)
    a, b, Z0, ok = O.acoustic_coefficients(cfg, w["h"], w["dt"], w["P0"], w["rho"], w["c"])
    assert ok
    p = O.scale_pressure(w["p0"], w["P0"], sfmt).reshape(w["p0"].shape)
    vs = [O.scale_velocity(v0[ax], Z0, w["P0"], sfmt).reshape(w["p0"].shape) for ax in range(3)]
    del w["rho"], w["c"], w["p0"], v0
    n = 512
    rng = np.random.default_rng(11)
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1), (n // 2, n // 2, n // 2), (n // 2 + 1, n // 2 - 3, n // 2 + 2),
           (0, n // 2, n // 2), (n - 1, 5, n - 2), (63, 64, 65), (64, 63, 1), (1, 1, n - 1),
           (n - 8, n // 2 + 7, 0), (7, 8, 9), (n - 9, n - 17, 128)]
    pts += [tuple(int(x) for x in rng.integers(0, n, 3)) for _ in range(20)]
    expect = _subbox_expect({"shape": (n, n, n)}, {"a": a, "b": b, "p": p, "v": vs}, prec, comp, steps, pts)
    bad = []
    for (i, j, k), ex in zip(pts, expect):
        for key, val in ex.items():
            if key not in got:
                continue
            g = got[key][k, j, i]
            r = to_bits(np.array([val]), sfmt)[0]
            if g != r:
                bad.append(f"{key} at {(i, j, k)}: gpu {g:#x} oracle {r:#x}")
    assert not bad, bad[:10]
    # the sampled field is not trivially zero
    assert np.count_nonzero(got["p"]) > 1000
    assert sum(1 for ex in expect if ex["p"] != 0) > len(pts) // 2


# ------------------------------------------------------ one-pass step (fused)
FUSED_VARIANTS = VARIANTS


def _uniform_rho_run(shape, bc, prec, comp, steps, zchunk, src=False, energy=True, seed=0):
    """The one-pass step needs a uniform density; the sound speed varies."""
    h = 10.0
    c = inputs.smooth_random_field(shape, seed, 3.0, 1500.0, 4500.0)
    rho = np.full(c.shape, 1000.0)
    dt = 0.4 * h / 4500.0 / np.sqrt(1.5)
    p0 = inputs.gaussian(shape, h, 3.0 * h)
    rng = np.random.default_rng(seed)
    p0 = p0 + 0.2 * rng.standard_normal(p0.shape)
    v0 = [0.1 / 4.5e6 * rng.standard_normal(p0.shape) for _ in range(3)]
    s = None
    if src:
        wav = inputs.ricker_table(steps, dt, 40.0) * 0.5 * h * h / 4.5e6
        s = ([shape[0] // 2 + 3, shape[1] // 3, shape[2] // 2], wav)
    ctx, st = acoustic_pair(shape, bc, prec, comp, h, dt, rho, c, p0=p0, v0=v0, src=s,
                            zchunk=zchunk, kernel=3)
    try:
        W.wave_set_timing(ctx, True)
        W.wave_step(ctx, steps)
        nl, _ = W.wave_get_timing(ctx, 3)
        assert nl == steps, "the one-pass kernel did not run"
        _, E = st.run(steps, energy=energy)
        bad = compare_acoustic(ctx, st, prec, comp)
        if energy:
            e_gpu = W.wave_energy(ctx)
            e_orc = E[-1] * O.energy_factor(h, dt, 1.0, st.Z0, 3)
            if not abs(e_gpu - e_orc) <= 2e-6 * abs(e_orc):
                bad.append(f"energy {e_gpu} vs oracle {e_orc}")
        W.wave_sync(ctx)
    finally:
        W.wave_destroy(ctx)
    assert not bad, bad


@pytest.mark.parametrize("prec,comp", FUSED_VARIANTS)
def test_fused_ragged_y_z_rigid_many_chunks(prec, comp):
    nx = 128 if prec != "fp32" else 64
    _uniform_rho_run((nx, 37, 29), (R, R, R), prec, comp, 7, zchunk=5)


@pytest.mark.parametrize("ny", [8, 17, 19, 34, 50])
def test_fused_rigid_y_faces_every_tail(ny):
    """Rigid y walls: the tiles at the y faces load whole boxes (rows past the
    faces read as zero) and take the images from the mirror rows inside the
    tile. Row counts that leave 1, 2, 3 and 16 rows in the last tile, and one
    tile spanning both faces."""
    _uniform_rho_run((64, ny, 11), (R, R, R), "fp16", 3, 9, zchunk=4, src=True)
    _uniform_rho_run((32, ny, 9), (R, R, P), "fp32", 0, 6, zchunk=3)
    _uniform_rho_run((64, ny, 10), (R, R, P), "fp16_pairs", 3, 7, zchunk=3, src=True)


@pytest.mark.parametrize("prec,comp", [("fp16", 3), ("bf16", 6), ("fp32", 0), ("fp16_f32arith", 3),
                                       ("fp16_pairs", 3)])
def test_fused_periodic_mixed_source(prec, comp):
    """Periodic y and z, rigid x (the one-pass step reads rigid x images)."""
    nx = 192 if prec != "fp32" else 96
    _uniform_rho_run((nx, 20, 17), (R, P, P), prec, comp, 6, zchunk=4, src=True)
    _uniform_rho_run((nx, 33, 40), (R, P, R), prec, comp, 5, zchunk=32, src=True)
    _uniform_rho_run((nx, 16, 9), (R, R, P), prec, comp, 9, zchunk=3)
    _uniform_rho_run((64 if prec != "fp32" else 32, 8, 8), (R, R, R), prec, comp, 11, zchunk=8)


def test_fused_request_with_periodic_x_falls_back_bit_exact():
    """kernel=3 with periodic x faces runs the two-kernel step, still bit-exact."""
    _run((128, 20, 17), (P, P, P), "fp16", 3, 6, zchunk=4, src=True, energy=True, kernel=3)
