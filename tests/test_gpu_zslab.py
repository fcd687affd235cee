"""Z slabs on the GPU (domain decomposition along z; not in the paper): a 3D
acoustic grid split into slab contexts on one GPU, stepped by half steps with
the ghost planes exchanged in between (paper_2310_00236_gb300.zslab), gives
bit for bit the whole grid's values, which equal the oracle's. The slabs run
one after the other on one stream and exchange by device copies; no kernel
waits for another."""
import numpy as np
import pytest

import oracle as O
from paper_2310_00236_gb300 import inputs, zslab
from paper_2310_00236_gb300 import wave as W
from wave_helpers import PREC, acoustic_pair, compare_acoustic, gpu_bits, to_bits

pytestmark = pytest.mark.gpu


def _problem(shape, seed):
    nx, ny, nz = shape
    h = 10.0
    c = inputs.smooth_random_field(shape, seed, 2.0, 1500.0, 4500.0)
    rho = inputs.smooth_random_field(shape, seed + 1, 2.0, 1000.0, 2600.0)
    dt = 0.4 * h / 4500.0
    rng = np.random.default_rng(seed)
    p0 = inputs.gaussian(shape, h, 40.0) + 0.05 * rng.standard_normal(c.shape)
    return h, dt, rho, c, p0


@pytest.mark.parametrize("prec,comp,nslabs", [("fp16", 3, 2), ("fp16", 0, 3), ("bf16", 6, 2),
                                              ("fp32", 0, 2), ("fp16_f32arith", 3, 3)])
def test_slabs_equal_whole_grid_and_oracle(prec, comp, nslabs):
    import torch
    shape = (48, 20, 33)
    steps = 14
    h, dt, rho, c, p0 = _problem(shape, 3)
    code = PREC[prec][0]
    # physical amplitude whose scaled increment b s^ stays near 0.1 (s^ = w Z0 / h^2)
    wav = np.sin(np.arange(steps) * 0.6) * 0.25 * h * h / float(rho.max() * c.max())
    src = (11, 9, 25)
    # the whole grid on the same (streaming) kernels, and the oracle
    ctx, st = acoustic_pair(shape, (1, 1, 1), prec, comp, h, dt, rho, c, p0=p0, src=(list(src), wav), kernel=2)
    slabs = []
    try:
        W.wave_step(ctx, steps)
        e_whole = W.wave_energy(ctx)
        st.run(steps)
        assert not compare_acoustic(ctx, st, prec, comp)
        bounds = [zslab.slab_bounds(shape[2], nslabs, r) for r in range(nslabs)]
        for z0, z1 in bounds:
            s = zslab.Slab(shape, z0, z1, h, rho, c, dt, code, comp)
            W.wave_set_initial(s.ctx, W.WAVE_F_P, p0[z0:z1])
            if z0 <= src[2] < z1:
                W.wave_set_source(s.ctx, W.WAVE_F_P, [src[0], src[1], src[2] - z0], wav)
            slabs.append(s)
        zslab.exchange_local(slabs, "p")
        for _ in range(steps):
            for s in slabs:
                s.half_step(0)
            zslab.exchange_local(slabs, "vz")
            for s in slabs:
                s.half_step(1)
            zslab.exchange_local(slabs, "p")
        torch.cuda.synchronize()
        bad = []
        for fid in (W.WAVE_F_P, W.WAVE_F_VX, W.WAVE_F_VY, W.WAVE_F_VZ):
            for t in ((0, 1) if comp else (0,)):
                whole = gpu_bits(W.wave_get_raw(ctx, fid, t))
                parts = np.concatenate([gpu_bits(W.wave_get_raw(s.ctx, fid, t)) for s in slabs])
                if not np.array_equal(whole, parts):
                    bad.append((fid, t, int(np.count_nonzero(whole != parts))))
        assert not bad, bad
        # the multipliers of each slab are the whole grid's planes (shared Z0,
        # density averaged across the cuts)
        for k in range(4):
            whole, z_whole = W.wave_get_coefficient(ctx, k)
            for s in slabs:
                part, z_part = W.wave_get_coefficient(s.ctx, k)
                assert z_part == z_whole
                np.testing.assert_array_equal(part, whole[s.z0:s.z1])
        e_parts = sum(W.wave_energy(s.ctx) for s in slabs)
        assert abs(e_parts - e_whole) <= 1e-9 * abs(e_whole)
    finally:
        W.wave_destroy(ctx)
        for s in slabs:
            s.destroy()


def test_slab_call_order_and_ghost_checks():
    import torch
    shape = (32, 16, 24)
    h, dt, rho, c, p0 = _problem(shape, 5)
    s = zslab.Slab(shape, 0, 12, h, rho, c, dt, W.WAVE_FP16, 3)
    try:
        with pytest.raises(W.WaveError) as e:
            W.wave_step(s.ctx, 1)                       # slabs take half steps
        assert e.value.status == W.WAVE_ESTATE
        with pytest.raises(W.WaveError) as e:
            W.wave_half_step(s.ctx, 1)                  # velocities first
        assert e.value.status == W.WAVE_ESTATE
        g = torch.zeros(2 * W.wave_get_layout(s.ctx)[1], dtype=torch.int16, device="cuda")
        with pytest.raises(W.WaveError) as e:
            W.wave_set_z_ghosts(s.ctx, g, g, g, g)      # the z-lo face is the grid's wall
        assert e.value.status == W.WAVE_EINVAL
        one_plane = g[: W.wave_get_layout(s.ctx)[1]]
        with pytest.raises(ValueError):                 # refused by the binding, before the library
            W.wave_set_z_ghosts(s.ctx, None, one_plane, None, one_plane)
        with pytest.raises(ValueError):
            W.wave_copy_planes(s.ctx, W.WAVE_F_P, 0, 2, one_plane)
        W.wave_half_step(s.ctx, 0)
        with pytest.raises(W.WaveError) as e:
            W.wave_half_step(s.ctx, 0)                  # the pressure half is due
        assert e.value.status == W.WAVE_ESTATE
        W.wave_half_step(s.ctx, 1)
        with pytest.raises(W.WaveError) as e:
            W.wave_copy_planes(s.ctx, W.WAVE_F_P, 11, 2, g)   # past the slab
        assert e.value.status == W.WAVE_EINVAL
    finally:
        s.destroy()
