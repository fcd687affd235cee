"""The allocation-free energy entry point (wave_energy_acoustic_static).

It exists for callers that cannot call cudaMalloc, such as a host framework
that reserves the whole device heap at start-up and hands out only views of
it, or a real-time loop whose memory budget forbids allocating after start-up.
It takes the fields and multipliers the caller already holds on the device and
keeps its reduction scratch in a fixed static device array.

This test runs an ordinary context (3D and 2D), reads back p^n, p^{n+1},
v^{n+1/2} and the multipliers of its last step, and checks that the static
entry point returns the energy wave_energy reported, on two calls in a row
(the second call finds the static array as the first left it). It lives in
its own file so that it is collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2310_00236_gb300 import inputs
from paper_2310_00236_gb300 import wave as W

pytestmark = pytest.mark.gpu


def _device_raw(torch, arr):
    a = np.ascontiguousarray(arr)
    if a.dtype == np.uint16:
        return torch.from_numpy(a.view(np.int16).copy()).cuda()
    return torch.from_numpy(a.astype(np.float32)).cuda()


def _coef_raw(coef, prec):
    if prec == W.WAVE_FP32:
        return coef.astype(np.float32)
    if prec == W.WAVE_BF16:
        import torch
        return torch.from_numpy(coef.astype(np.float32)).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    return coef.astype(np.float16).view(np.uint16)


@pytest.mark.parametrize("shape", [(64, 40, 36), (130, 97)])
@pytest.mark.parametrize("prec", [W.WAVE_FP16, W.WAVE_BF16, W.WAVE_FP32])
def test_static_energy_matches_wave_energy_twice(prec, shape):
    import torch
    nd = len(shape)
    h = 10.0
    c = inputs.smooth_random_field(shape, 1, 3.0, 1500.0, 4500.0)
    rho = inputs.smooth_random_field(shape, 2, 3.0, 1000.0, 2600.0)
    dt = 0.4 * h / 4500.0 / np.sqrt(nd / 2.0)
    rng = np.random.default_rng(0)
    p0 = inputs.gaussian(shape, h, 30.0) + 0.1 * rng.standard_normal(c.shape)
    ctx = W.wave_create(shape, h, rho, c, dt, prec, W.WAVE_COMP_3OP, bc=[W.WAVE_BC_RIGID] * 2 * nd
                        + [W.WAVE_BC_PERIODIC] * (6 - 2 * nd))
    try:
        W.wave_set_initial(ctx, W.WAVE_F_P, p0)
        results = []
        for call in range(2):
            W.wave_step(ctx, 4 + call)
            p_old = W.wave_get_raw(ctx, W.WAVE_F_P)
            W.wave_step(ctx, 1)
            e_ref = W.wave_energy(ctx)
            p_new = W.wave_get_raw(ctx, W.WAVE_F_P)
            v = [W.wave_get_raw(ctx, W.WAVE_F_VX + d) for d in range(nd)]
            b, z0 = W.wave_get_coefficient(ctx, 0)
            a = [W.wave_get_coefficient(ctx, 1 + d)[0] for d in range(nd)]
            factor = 0.5 * h ** (nd - 1) * 1.0 * 1.0 * dt / z0
            out = torch.zeros(1, dtype=torch.float64, device="cuda")
            W.wave_energy_acoustic_static(
                nd, shape, prec, _device_raw(torch, p_old), _device_raw(torch, p_new),
                [_device_raw(torch, x) for x in v],
                [_device_raw(torch, _coef_raw(x, prec)) for x in a],
                _device_raw(torch, _coef_raw(b, prec)), factor, out)
            torch.cuda.synchronize()
            e_static = float(out.item())
            results.append(e_static)
            assert abs(e_static - e_ref) <= 2e-6 * abs(e_ref), (call, e_static, e_ref)
        assert results[0] != results[1]       # two different states, both right
    finally:
        W.wave_destroy(ctx)


def test_static_energy_rejects_sizes_beyond_its_scratch():
    """Called through the C ABI directly (the binding would already refuse
    arrays smaller than the grid): grids above the static array's limit, and
    extents whose product overflows, come back as WAVE_EINVAL before any
    device work."""
    import torch
    lib = W.lib()
    t = torch.zeros(8, dtype=torch.int16, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    ptr = C.c_void_p(t.data_ptr())
    arr = (C.c_void_p * 3)(t.data_ptr(), t.data_ptr(), t.data_ptr())
    for n in ((512, 512, 65), (1 << 40, 1 << 40, 1 << 40), (1 << 62, 4, 4)):
        nn = (C.c_int64 * 3)(*n)
        st = lib.wave_energy_acoustic_static(3, nn, W.WAVE_FP16, ptr, ptr, arr, arr, ptr, C.c_double(1.0),
                                             C.c_void_p(out.data_ptr()), None)
        assert st == W.WAVE_EINVAL, n
        assert b"static scratch limit" in lib.wave_last_error()
