"""GPU parity of the batched multi-shot 2D path.

A batch advances many independent 2D acoustic problems with the same launches.
Every shot must carry exactly the bits it carries when stepped alone through
wave_step (the one-problem path, itself bit-exact against the oracle), and one
shot per case is also compared with the oracle directly. The cases cover
ragged grid sizes (tiles cut by both edges, grids smaller than one tile), each
shot's own source and medium, the autotuned launch shapes and CUDA-graph
replays of step runs, and calls that continue a batch.
"""
import numpy as np
import pytest

import oracle as O
from paper_2310_00236_gb300 import inputs
from paper_2310_00236_gb300 import wave as W
from wave_helpers import PREC, acoustic_pair, compare_acoustic, gpu_bits

pytestmark = pytest.mark.gpu
R, P = W.WAVE_BC_RIGID, W.WAVE_BC_PERIODIC


def _shot(shape, bc, prec, comp, seed, nsteps, stream=None, kernel=0):
    """One seeded shot: smooth random velocity in [1500, 4500], a Gaussian
    initial pressure and a Ricker source. Returns (ctx, oracle state)."""
    nx, ny = shape
    h = 10.0
    c = inputs.smooth_random_field((nx, ny), seed, max(2.0, nx / 32), 1500.0, 4500.0)
    rho = np.full((ny, nx), 1000.0)
    dt = 0.4 * h / 4500.0
    P0 = 1e5
    p0 = P0 * inputs.gaussian(shape, 1.0 / max(nx, ny), 0.1)
    z0 = 1000.0 * float(c.max())
    wav = 0.5 * P0 * h / z0 * inputs.ricker_table(nsteps, dt, 1.0 / (30 * dt))
    src = ([nx // 2, min(8, ny - 1)], wav)
    return acoustic_pair(shape, bc, prec, comp, h, dt, rho, c, p0=p0, P0=P0, src=src, stream=stream,
                         kernel=kernel)


def _fields(ctx, comp):
    out = []
    for fid in (W.WAVE_F_P, W.WAVE_F_VX, W.WAVE_F_VY):
        out.append(gpu_bits(W.wave_get_raw(ctx, fid, 0)))
        if comp:
            out.append(gpu_bits(W.wave_get_raw(ctx, fid, 1)))
    return out


def _run_case(shapes, bcs, prec, comp, calls, stream=None, oracle_shot=0, kernel=0, shape=None):
    """Batch the shots and step them by the step counts in `calls`; step twin
    contexts (default kernels) one by one; compare bits and energies.
    kernel = 3: the batched contexts keep the second buffer set, so the tuner
    also tries the one-pass strips."""
    total = sum(calls)
    pairs = [_shot(s, b, prec, comp, 100 + i, total, stream, kernel) for i, (s, b) in enumerate(zip(shapes, bcs))]
    twins = [_shot(s, b, prec, comp, 100 + i, total, stream)[0] for i, (s, b) in enumerate(zip(shapes, bcs))]
    ctxs = [p[0] for p in pairs]
    batch = W.wave_batch_create(ctxs)
    if shape is not None:
        W.wave_batch_set_shape(batch, shape)
    try:
        for n in calls:
            W.wave_batch_step(batch, n)
            for t in twins:
                W.wave_step(t, n)
        bad = []
        for i, (c, t) in enumerate(zip(ctxs, twins)):
            for k, (g, r) in enumerate(zip(_fields(c, comp), _fields(t, comp))):
                if not np.array_equal(g, r):
                    bad.append(f"shot {i} {shapes[i]} array {k}: {int(np.count_nonzero(g != r))} mismatches")
            eb, et = W.wave_energy(c), W.wave_energy(t)
            if not abs(eb - et) <= 1e-12 * abs(et):
                bad.append(f"shot {i} energy {eb} vs {et}")
        st = pairs[oracle_shot][1]
        _, E = st.run(total, energy=True)
        bad += [f"oracle shot {oracle_shot}: {m}" for m in compare_acoustic(ctxs[oracle_shot], st, prec, comp)]
        h, dt = 10.0, 0.4 * 10.0 / 4500.0
        e_orc = E[-1] * O.energy_factor(h, dt, 1e5, st.Z0, 2)
        # the kernels form each energy term in binary32 (one rounded product
        # for fp32 fields, one rounded division): relative error <= 2^-23 per
        # term, against the oracle's binary64 terms
        if not abs(W.wave_energy(ctxs[oracle_shot]) - e_orc) <= 1e-6 * abs(e_orc):
            bad.append(f"oracle energy {W.wave_energy(ctxs[oracle_shot])} vs {e_orc}")
        info = W.wave_batch_info(batch)
    finally:
        W.wave_batch_destroy(batch)
        for c in ctxs + twins:
            W.wave_destroy(c)
    assert not bad, bad[:10]
    return info


SHAPES = [(37, 29), (64, 48), (100, 33), (8, 8), (129, 70)]
BCS = [(R, R), (P, R), (R, P), (R, R), (P, P)]


@pytest.mark.parametrize("prec,comp", [("fp16", 3), ("fp16", 0), ("bf16", 6), ("fp32", 0),
                                       ("fp16_f32arith", 3), ("fp16_pairs", 3)])
def test_batch_bit_exact_ragged_shots(prec, comp):
    _run_case(SHAPES, BCS, prec, comp, [12])


def test_batch_autotune_and_graph_replay():
    import torch
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        info = _run_case(SHAPES[:3], BCS[:3], "fp16", 3, [100, 40, 1, 7], stream=stream.cuda_stream,
                         oracle_shot=2)
    assert info["tuned"]
    assert info["threads"] % 32 == 0
    # the two-launch kinds replay graphs of 32 steps; the persistent kind runs
    # every step of a call in one cooperative launch
    if info["kind"] == "persistent strips":
        assert info["graph_steps"] == 0
    else:
        assert info["blocks"] > 0 and info["graph_steps"] == 32


@pytest.mark.parametrize("prec,comp", [("fp16", 3), ("fp32", 0)])
def test_batch_one_pass_candidates_bit_exact(prec, comp):
    """Contexts with the second buffer set: the tuner runs all 24 launch
    shapes (the one-pass strips last), the state follows the buffer sets
    through odd and even step counts, and every shot equals its twin stepped
    alone by the two-launch strips."""
    import torch
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        info = _run_case(SHAPES, BCS, prec, comp, [27, 40, 1, 7, 33], stream=stream.cuda_stream,
                         oracle_shot=4, kernel=3)
    assert info["tuned"]


def test_batch_default_stream_tuned_without_graph():
    info = _run_case(SHAPES[:2], BCS[:2], "fp16", 6, [60], oracle_shot=1)
    assert info["tuned"] and info["graph_steps"] == 0


def test_batch_single_shot_equals_oracle():
    _run_case([(256, 200)], [(R, R)], "fp16", 3, [30])


def test_batch_rejects_mixed_contexts():
    a, _ = _shot((32, 16), (R, R), "fp16", 3, 1, 4)
    b, _ = _shot((32, 16), (R, R), "bf16", 3, 2, 4)
    c3 = W.wave_create((16, 8, 8), 1.0, np.ones((8, 8, 16)), np.ones((8, 8, 16)), 0.1, W.WAVE_FP16, 3)
    try:
        for bad in ([a, b], [a, c3], [a, a]):
            with pytest.raises(W.WaveError) as ei:
                W.wave_batch_create(bad)
            assert ei.value.status == W.WAVE_EINVAL
    finally:
        for c in (a, b, c3):
            W.wave_destroy(c)


@pytest.mark.parametrize("prec,comp", [("fp16", 3), ("fp32", 0), ("bf16", 6), ("fp16_pairs", 3)])
@pytest.mark.parametrize("shape", [14, 17])
def test_batch_persistent_launch_bit_exact(prec, comp, shape):
    """The persistent kind (every step of a call in one cooperative launch,
    grid barriers between the half steps): every shot equals its twin stepped
    alone, over calls of several lengths, one shot equals the oracle, and the
    per-shot energies agree."""
    import torch
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        info = _run_case(SHAPES, BCS, prec, comp, [30, 1, 7, 64], stream=stream.cuda_stream, oracle_shot=3,
                         shape=shape)
    assert info["kind"] == "persistent strips" and info["graph_steps"] == 0
