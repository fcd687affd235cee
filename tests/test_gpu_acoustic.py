"""GPU parity of the acoustic path against the CPU oracle (bit-exact).

Every field and every compensation array of the CUDA path must equal the
oracle's op-by-op emulation bit for bit, for every precision and update
variant, on grids that span several thread blocks with ragged tails, with
both boundary kinds, variable media, a point source and receivers.
"""
import numpy as np
import pytest

import oracle as O
from paper_2310_00236_gb300 import inputs
from paper_2310_00236_gb300 import wave as W
from wave_helpers import PAIRS, PREC, acoustic_pair, compare_acoustic

pytestmark = pytest.mark.gpu

VARIANTS = [("fp16", 0), ("fp16", 3), ("fp16", 6), ("bf16", 0), ("bf16", 3), ("bf16", 6),
            ("fp32", 0), ("fp32", 3), ("fp16_f32arith", 0), ("fp16_f32arith", 3),
            ("bf16_f32arith", 3), ("fp16_pairs", 3)]
# (kernel, precision, compensation); the one-pass strips read stored values only
KVARIANTS = [(k, p, c) for k in (4, 1, 2, 3) for p, c in VARIANTS if not (k == 3 and p in PAIRS)]


def _media(shape, seed, h):
    c = inputs.smooth_random_field(shape, seed, 3.0, 1500.0, 4500.0)
    rho = inputs.smooth_random_field(shape, seed + 1, 3.0, 1000.0, 2600.0)
    return rho, c


def _run(shape, bc, prec, comp, steps, seed=0, variable=True, src=False, kernel=0):
    nd = len(shape)
    h = 10.0
    if variable:
        rho, c = _media(shape, seed, h)
    else:
        rho = np.full(tuple(shape[::-1]), 1000.0)
        c = np.full(tuple(shape[::-1]), 3000.0)
    dt = 0.4 * h / 4500.0 / np.sqrt(nd / 2.0)
    p0 = inputs.gaussian(shape, h, 2.5 * h)
    rng = np.random.default_rng(seed)
    v0 = [1e-4 * rng.standard_normal(p0.shape) for _ in range(nd)]
    s = None
    if src:
        # amplitude chosen so the scaled source w Z0 / (P0 h^(d-1)) is about 0.5
        z0 = float(np.max(rho) * np.max(c))
        wav = inputs.ricker_table(steps, dt, 40.0) * 0.5 * h ** (nd - 1) / z0
        s = ([shape[a] // 3 for a in range(nd)], wav)
    ctx, st = acoustic_pair(shape, bc, prec, comp, h, dt, rho, c, p0=p0, v0=v0, src=s,
                            kernel=kernel)
    try:
        W.wave_step(ctx, steps)
        st.run(steps)
        bad = compare_acoustic(ctx, st, prec, comp)
    finally:
        W.wave_destroy(ctx)
    assert not bad, bad


R, P = O.BC_RIGID, O.BC_PERIODIC


# kernel 4 (the default for small grids): cluster-resident steps (the whole
# state in one cluster's shared memory, bands of rows per CTA, rows past a band
# read from the neighbouring CTA); kernel 1: one thread per point; kernel 2:
# row strips, one launch per half step; kernel 3: one-pass row strips (both
# half steps in one launch, two buffer sets)
@pytest.mark.parametrize("kernel,prec,comp", KVARIANTS)
def test_2d_bit_exact_ragged_rigid(prec, comp, kernel):
    _run((37, 29), (R, R), prec, comp, 30, kernel=kernel)


@pytest.mark.parametrize("kernel,prec,comp", KVARIANTS)
def test_2d_bit_exact_periodic_source(prec, comp, kernel):
    _run((64, 40), (P, P), prec, comp, 25, src=True, kernel=kernel)


@pytest.mark.parametrize("kernel", [4, 2, 3])
@pytest.mark.parametrize("shape", [(257, 33), (300, 70), (8, 200), (513, 9), (265, 40), (520, 17)])
def test_2d_strips_ragged_wide_and_tall(shape, kernel):
    # strips of 256 points (128 for binary32) cut by the grid's x extent, rows
    # cut by the 16-row items, periodic x wrapping across strip boundaries;
    # the one-pass strips also recompute the x neighbours of v_x at strip
    # edges (from the neighbouring vectors, or point by point near the faces)
    _run(shape, (P, R), "fp16", 3, 12, src=True, kernel=kernel)
    _run(shape, (R, P), "fp32", 0, 12, kernel=kernel)
    _run(shape, (R, R), "bf16", 6, 11, src=True, kernel=kernel)
    if kernel != 3:
        # pair taps: the t queues and x neighbours of t follow the same paths
        _run(shape, (P, R), "fp16_pairs", 3, 12, src=True, kernel=kernel)


@pytest.mark.parametrize("prec,comp", [("fp16", 3), ("bf16", 6), ("fp32", 0),
                                       ("fp16_f32arith", 3), ("fp16_pairs", 6)])
def test_2d_mixed_bc_minimum_size(prec, comp):
    _run((8, 8), (R, P), prec, comp, 40)
    _run((9, 8), (P, R), prec, comp, 40, variable=False)


@pytest.mark.parametrize("prec,comp", VARIANTS)
def test_3d_bit_exact(prec, comp):
    _run((21, 18, 13), (R, P, R), prec, comp, 12)


@pytest.mark.parametrize("prec,comp", [("fp16", 3), ("fp32", 0), ("bf16", 0), ("fp16_pairs", 3)])
def test_3d_bit_exact_larger_source(prec, comp):
    _run((70, 36, 24), (R, R, R), prec, comp, 8, src=True)


def test_coefficients_bit_exact_and_uniform():
    shape = (33, 20, 12)
    rho, c = _media(shape, 3, 10.0)
    for prec in ("fp16", "bf16", "fp32", "fp16_pairs"):
        code, sfmt, _ = PREC[prec]
        if prec in PAIRS:
            sfmt = O.FP32      # the pair precision keeps the multipliers in binary32
        dt = 0.4 * 10.0 / 4500.0 / np.sqrt(1.5)
        ctx = W.wave_create(shape, 10.0, rho, c, dt, code, 3, bc=[1] * 6)
        cfg = O.acoustic_cfg(shape, (R, R, R), sfmt, 3)
        a, b, Z0, ok = O.acoustic_coefficients(cfg, 10.0, dt, 1.0, rho, c)
        assert ok
        try:
            gb, gz0 = W.wave_get_coefficient(ctx, 0)
            assert gz0 == Z0
            assert np.array_equal(gb, b)
            for ax in range(3):
                ga, _ = W.wave_get_coefficient(ctx, 1 + ax)
                assert np.array_equal(ga, a[ax])
        finally:
            W.wave_destroy(ctx)


def test_energy_matches_oracle_and_is_conserved_fp32():
    shape = (48, 40)
    h = 1.0 / 48
    w = inputs.acoustic_2d_gaussian(48, 200)
    ctx, st = acoustic_pair(shape, (R, R), "fp32", 0, h, 0.5 * h, w["rho"][:40, :48],
                            w["c"][:40, :48], p0=inputs.gaussian(shape, h, 0.1))
    try:
        import torch
        tr = torch.zeros(200, dtype=torch.float64, device="cuda")
        W.wave_set_energy_trace(ctx, tr, 200)
        W.wave_step(ctx, 200)
        _, E = st.run(200, energy=True)
        fac = O.energy_factor(h, 0.5 * h, 1.0, st.Z0, 2)
        Eg = tr.cpu().numpy()
        np.testing.assert_allclose(Eg, E * fac, rtol=2e-6)
        assert W.wave_energy(ctx) == Eg[-1]
        assert np.max(np.abs(Eg - Eg[0])) / Eg[0] < 1e-5
    finally:
        W.wave_destroy(ctx)


def test_receivers_match_oracle_traces():
    import torch
    shape = (40, 36)
    h = 5.0
    rho, c = _media(shape, 9, h)
    dt = 0.4 * h / 4500.0
    steps = 50
    wav = inputs.ricker_table(steps, dt, 30.0) * 0.5 * h / float(np.max(rho) * np.max(c))
    recs = [(5, 7), (20, 30), (39, 35), (0, 0)]
    ctx, st = acoustic_pair(shape, (R, P), "fp16", 3, h, dt, rho, c, src=([13, 11], wav))
    try:
        tr = torch.zeros(steps * len(recs), dtype=torch.float32, device="cuda")
        W.wave_set_receivers(ctx, W.WAVE_F_P, recs, tr, steps)
        W.wave_step(ctx, steps)
        ridx = [int(np.ravel_multi_index((j, i), st.shape)) for i, j in recs]
        traces, _ = st.run(steps, rec_field=0, rec_index=ridx)
        got = tr.cpu().numpy().reshape(steps, len(recs)).astype(np.float64)
        assert np.array_equal(got, traces)
        assert np.any(got != 0)
    finally:
        W.wave_destroy(ctx)


def test_state_roundtrip_resume_is_bit_exact():
    shape = (30, 26)
    h = 10.0
    rho, c = _media(shape, 4, h)
    dt = 0.4 * h / 4500.0
    p0 = inputs.gaussian(shape, h, 30.0)
    ctx, _ = acoustic_pair(shape, (R, R), "fp16", 3, h, dt, rho, c, p0=p0)
    ctx2, _ = acoustic_pair(shape, (R, R), "fp16", 3, h, dt, rho, c, p0=p0)
    try:
        W.wave_step(ctx, 10)
        blob = W.wave_get_state(ctx)
        W.wave_step(ctx, 15)
        W.wave_set_state(ctx2, blob)
        assert W.wave_steps_done(ctx2) == 10
        W.wave_step(ctx2, 15)
        for f in (W.WAVE_F_P, W.WAVE_F_VX, W.WAVE_F_VY):
            for cflag in (0, 1):
                assert np.array_equal(W.wave_get_raw(ctx, f, cflag), W.wave_get_raw(ctx2, f, cflag))
    finally:
        W.wave_destroy(ctx)
        W.wave_destroy(ctx2)


def test_runs_are_deterministic():
    shape = (45, 33, 20)
    for _ in range(1):
        rho, c = _media(shape, 2, 10.0)
        outs = []
        for rep in range(2):
            ctx, _ = acoustic_pair(shape, (R, R, R), "fp16", 3, 10.0, 0.4 * 10 / 4500 / 1.22,
                                   rho, c, p0=inputs.gaussian(shape, 10.0, 25.0))
            W.wave_step(ctx, 20)
            outs.append((W.wave_get_raw(ctx, W.WAVE_F_P), W.wave_energy(ctx)))
            W.wave_destroy(ctx)
        assert np.array_equal(outs[0][0], outs[1][0])
        assert outs[0][1] == outs[1][1]


def test_acoustic2d_256_full_size_2000_steps_bit_exact():
    """2D acoustic 256^2, rho = c = 1, p = 0 walls, Gaussian, CFL 0.5, 2000
    steps, fp16 + sum_3op: every stored bit equals the oracle's."""
    w = inputs.acoustic_2d_gaussian(256, 2000)
    ctx, st = acoustic_pair(w["shape"], (R, R), "fp16", 3, w["h"], w["dt"], w["rho"], w["c"],
                            p0=w["p0"])
    try:
        W.wave_step(ctx, 2000)
        st.run(2000)
        bad = compare_acoustic(ctx, st, "fp16", 3)
    finally:
        W.wave_destroy(ctx)
    assert not bad, bad


def test_acoustic2d_256_pairs_full_size_bit_exact_and_within_2e3():
    """The same problem with the pair stencils (binary16 V and T, binary32
    registers, every tap RN32(V + T)): every stored bit equals the oracle's
    pair_stencil run, and the pressure is within 2e-3 relative L2 of the
    binary64 oracle run (fp16 + sum_3op with the stored-value stencil is not:
    about 1.4e-2)."""
    w = inputs.acoustic_2d_gaussian(256, 2000)
    ctx, st = acoustic_pair(w["shape"], (R, R), "fp16_pairs", 3, w["h"], w["dt"], w["rho"], w["c"],
                            p0=w["p0"])
    try:
        W.wave_step(ctx, 2000)
        st.run(2000)
        bad = compare_acoustic(ctx, st, "fp16_pairs", 3)
        p = W.wave_get_field(ctx, W.WAVE_F_P).reshape(st.p.shape)
    finally:
        W.wave_destroy(ctx)
    assert not bad, bad
    ref = O.acoustic_setup(w["shape"], (R, R), w["h"], w["dt"], w["rho"], w["c"], O.FP64, 0, p0=w["p0"])
    ref.run(2000)
    err = float(np.linalg.norm(p - ref.p * st.P0) / np.linalg.norm(ref.p * st.P0))
    assert err < 2e-3, err


def test_errors_reported_not_faulted():
    """Bad arguments come back as status codes, the context stays usable."""
    shape = (16, 16)
    ones = np.ones((16, 16))
    with pytest.raises(W.WaveError) as e:
        W.wave_create(shape, 0.1, ones, ones * 1e6, 0.1, W.WAVE_FP16, 3)
    assert e.value.status == W.WAVE_ERANGE          # b overflows binary16
    ctx = W.wave_create(shape, 0.1, ones, ones, 0.02, W.WAVE_FP16, 3)
    try:
        with pytest.raises(W.WaveError) as e:
            W.wave_energy(ctx)
        assert e.value.status == W.WAVE_ESTATE      # no step yet
        with pytest.raises(W.WaveError) as e:
            W.wave_set_initial(ctx, W.WAVE_F_P, np.full((16, 16), np.nan))
        assert e.value.status == W.WAVE_ERANGE
        with pytest.raises(W.WaveError) as e:
            W.wave_set_initial(ctx, W.WAVE_F_VZ, ones)
        assert e.value.status == W.WAVE_EINVAL
        with pytest.raises(W.WaveError) as e:
            W.wave_adjoint_step(ctx, 1)
        assert e.value.status == W.WAVE_ESTATE      # no recorded run
        W.wave_set_initial(ctx, W.WAVE_F_P, ones * 0.5)
        W.wave_step(ctx, 3)
        assert np.isfinite(W.wave_energy(ctx))
    finally:
        W.wave_destroy(ctx)


def test_2d_graph_replay_on_side_stream_bit_exact():
    """Plain 2D stepping on a created stream replays captured step graphs; the
    result equals the oracle, across calls and with a source."""
    import torch
    shape = (96, 70)
    h = 10.0
    rho, c = _media(shape, 5, h)
    dt = 0.4 * h / 4500.0
    z0 = float(np.max(rho) * np.max(c))
    steps = [70, 33, 5, 64]
    wav = inputs.ricker_table(sum(steps), dt, 40.0) * 0.5 * h / z0
    stream = torch.cuda.Stream()
    ctx, st = acoustic_pair(shape, (R, P), "fp16", 3, h, dt, rho, c,
                            p0=inputs.gaussian(shape, h, 2.5 * h), src=([30, 20], wav), stream=stream.cuda_stream,
                            kernel=2)
    try:
        for n in steps:
            W.wave_step(ctx, n)
        _, E = st.run(sum(steps), energy=True)
        bad = compare_acoustic(ctx, st, "fp16", 3)
        e_orc = E[-1] * O.energy_factor(h, dt, 1.0, st.Z0, 2)
        if not abs(W.wave_energy(ctx) - e_orc) <= 2e-6 * abs(e_orc):
            bad.append(f"energy {W.wave_energy(ctx)} vs {e_orc}")
    finally:
        W.wave_destroy(ctx)
    assert not bad, bad


@pytest.mark.parametrize("prec,comp", [("fp16", 3), ("fp32", 0), ("fp16_pairs", 3)])
def test_2d_cluster_receivers_and_energy_trace_across_calls(prec, comp):
    """Cluster-resident steps over several wave_step calls: the source's step
    index, the v_x receiver traces and the per-step energies continue across
    calls and stop at their capacities; fields, traces and energies equal the
    oracle's (energies to the binary32 terms' rounding)."""
    import torch
    shape = (150, 70)
    h = 10.0
    rho, c = _media(shape, 11, h)
    dt = 0.4 * h / 4500.0
    calls = [17, 1, 30]
    total = sum(calls)
    z0 = float(np.max(rho) * np.max(c))
    wav = inputs.ricker_table(total, dt, 40.0) * 0.5 * h / z0
    recs = [(5, 7), (75, 34), (149, 69), (0, 0), (140, 35)]
    cap_rec, cap_e = 40, 45
    ctx, st = acoustic_pair(shape, (R, P), prec, comp, h, dt, rho, c, p0=inputs.gaussian(shape, h, 3 * h),
                            src=([50, 35], wav), kernel=4)
    try:
        tr = torch.full((cap_rec * len(recs),), -7.0, dtype=torch.float32, device="cuda")
        en = torch.full((cap_e,), -7.0, dtype=torch.float64, device="cuda")
        W.wave_set_receivers(ctx, W.WAVE_F_VX, recs, tr, cap_rec)
        W.wave_set_energy_trace(ctx, en, cap_e)
        for n in calls:
            W.wave_step(ctx, n)
        ridx = [int(np.ravel_multi_index((j, i), st.shape)) for i, j in recs]
        traces, E = st.run(total, energy=True, rec_field=1, rec_index=ridx)
        bad = compare_acoustic(ctx, st, prec, comp)
        got = tr.cpu().numpy().reshape(cap_rec, len(recs)).astype(np.float64)
        if not np.array_equal(got, traces[:cap_rec]):
            bad.append("receiver traces differ")
        fac = O.energy_factor(h, dt, 1.0, st.Z0, 2)
        np.testing.assert_allclose(en.cpu().numpy(), E[:cap_e] * fac, rtol=2e-6)
        assert abs(W.wave_energy(ctx) - E[-1] * fac) <= 2e-6 * abs(E[-1] * fac)
        assert np.any(got != 0)
    finally:
        W.wave_destroy(ctx)
    assert not bad, bad


def test_2d_cluster_largest_grid_and_fit_limit():
    """512 x 448 binary16 + compensation (about 2.75 MB of state, 28 rows per
    band over 16 CTAs): bit-exact to the oracle and to the row strips; a grid
    whose state does not fit is refused by kernel 4 and stepped by the strips
    under kernel 0."""
    shape = (512, 448)
    h = 10.0
    rho, c = _media(shape, 12, h)
    dt = 0.4 * h / 4500.0
    p0 = inputs.gaussian(shape, h, 20 * h)
    ctx, st = acoustic_pair(shape, (R, R), "fp16", 3, h, dt, rho, c, p0=p0, kernel=4)
    twin, _ = acoustic_pair(shape, (R, R), "fp16", 3, h, dt, rho, c, p0=p0, kernel=2)
    try:
        W.wave_step(ctx, 30)
        W.wave_step(twin, 30)
        st.run(30)
        bad = compare_acoustic(ctx, st, "fp16", 3)
        for f in (W.WAVE_F_P, W.WAVE_F_VX, W.WAVE_F_VY):
            for cf in (0, 1):
                if not np.array_equal(W.wave_get_raw(ctx, f, cf), W.wave_get_raw(twin, f, cf)):
                    bad.append(f"field {f} comp {cf}: cluster and strips differ")
    finally:
        W.wave_destroy(ctx)
        W.wave_destroy(twin)
    assert not bad, bad
    big = (1024, 1024)
    ones = np.ones(big[::-1])
    with pytest.raises(W.WaveError) as e:
        W.wave_create(big, 1.0, ones, ones, 0.4, W.WAVE_FP16, 3, bc=[1] * 6, kernel=4)
    assert e.value.status == W.WAVE_EINVAL
    ctx = W.wave_create(big, 1.0, ones, ones, 0.4, W.WAVE_FP16, 3, bc=[1] * 6)
    try:
        W.wave_set_initial(ctx, W.WAVE_F_P, inputs.gaussian(big, 1.0, 30.0))
        W.wave_step(ctx, 3)
        assert np.isfinite(W.wave_energy(ctx))
    finally:
        W.wave_destroy(ctx)


def test_2d_default_kernel_choice():
    """Kernel 0 takes the cluster-resident steps (one launch per call) for a
    256^2 grid and the row strips (one launch sequence per step) for 384^2."""
    for side, launches in ((256, 1), (384, 10)):
        shape = (side, side)
        ones = np.ones(shape)
        ctx = W.wave_create(shape, 1.0 / side, ones, ones, 0.5 / side, W.WAVE_FP16, 3, bc=[1] * 6)
        try:
            W.wave_set_initial(ctx, W.WAVE_F_P, inputs.gaussian(shape, 1.0 / side, 0.05))
            W.wave_set_timing(ctx, True)
            W.wave_step(ctx, 10)
            n, _ = W.wave_get_timing(ctx, 3)
            assert n == launches, (side, n)
        finally:
            W.wave_destroy(ctx)


def test_bounded_wait_expiry_reports_timeout_and_leaves_gpu_usable():
    """A wait that nothing completes runs out, the host reads ETIMEOUT, the
    context is poisoned, and a new context on the same device steps normally."""
    shape = (16, 16)
    ones = np.ones((16, 16))
    ctx = W.wave_create(shape, 0.1, ones, ones, 0.02, W.WAVE_FP16, 3)
    try:
        with pytest.raises(W.WaveError) as e:
            W.wave_selftest_timeout(ctx)
        assert e.value.status == W.WAVE_ETIMEOUT
        with pytest.raises(W.WaveError) as e:
            W.wave_step(ctx, 1)
        assert e.value.status == W.WAVE_ESTATE
    finally:
        W.wave_destroy(ctx)
    ctx = W.wave_create(shape, 0.1, ones, ones, 0.02, W.WAVE_FP16, 3)
    try:
        W.wave_set_initial(ctx, W.WAVE_F_P, ones * 0.5)
        W.wave_step(ctx, 3)
        assert np.isfinite(W.wave_energy(ctx))
    finally:
        W.wave_destroy(ctx)
