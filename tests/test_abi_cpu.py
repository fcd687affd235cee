"""Host-side checks of the C ABI (no GPU needed): the library builds and
loads, it exports exactly the functions include/wave.h declares, and argument
errors are reported as status codes before any CUDA call is made."""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2310_00236_gb300 import build as B
from paper_2310_00236_gb300 import wave as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return W.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "wave.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"\b(wave_[a-z_]+)\s*\(", src)) - {"wave_alloc_fn", "wave_free_fn"}


def test_exports_match_header(lib):
    declared = _declared()
    assert declared == set(W.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (wave_[a-z_]+)$", out, flags=re.M))
    assert declared <= exported
    for name in declared:
        assert hasattr(lib, name)


def test_build_info(lib):
    assert "sm_103a" in W.wave_build_info()


def _ones(n=(16, 16)):
    return np.ones(n[::-1])


@pytest.mark.parametrize("kw,status", [
    (dict(n=(4, 16)), W.WAVE_EINVAL),                      # too small
    (dict(precision=W.WAVE_FP64), W.WAVE_ENOTIMPL),        # oracle only
    (dict(precision=17), W.WAVE_EINVAL),
    (dict(comp=4), W.WAVE_EINVAL),
    (dict(dt=-1.0), W.WAVE_EINVAL),
    (dict(dt=float("nan")), W.WAVE_EINVAL),
    (dict(spacing=(0.1, 0.2)), W.WAVE_EINVAL),             # anisotropic
    (dict(bc=(1, 0, 1, 1, 0, 0)), W.WAVE_EINVAL),          # mixed faces on one axis
    (dict(bc=(2, 2, 1, 1, 0, 0)), W.WAVE_EINVAL),          # free surface is elastic only
    (dict(field_scale=-1.0), W.WAVE_EINVAL),
    (dict(rho_scale=0.0), W.WAVE_ERANGE),                   # non-positive material
    (dict(kind=W.WAVE_ELASTIC, vs=True, n=(16, 16, 16)), W.WAVE_ENOTIMPL),   # elastic is 2D
    (dict(kind=W.WAVE_ELASTIC, vs=True, bc=(0, 1, 2, 1, 0, 0)), W.WAVE_EINVAL),  # mixed x faces
    (dict(kind=W.WAVE_ELASTIC, vs=True, bc=(2, 2, 2, 1, 0, 0)), W.WAVE_EINVAL),  # free x faces
    (dict(kind=W.WAVE_ELASTIC, vs=True, bc=(1, 1, 1, 2, 0, 0)), W.WAVE_EINVAL),  # free bottom
    (dict(kind=W.WAVE_ELASTIC, vs=False), W.WAVE_EINVAL),                        # no vs
    (dict(z_cut=1), W.WAVE_EINVAL),                          # z slabs are 3D
    (dict(z_cut=4, n=(16, 16, 16)), W.WAVE_EINVAL),          # bits 0 and 1 only
    (dict(z_cut=2, n=(16, 16, 16)), W.WAVE_EINVAL),          # a cut top face needs rho_above
    (dict(z_cut=1, kernel=3, n=(16, 16, 16)), W.WAVE_EINVAL),  # slabs use the streaming step
    (dict(z_cut=1, z0=-1.0, n=(16, 16, 16)), W.WAVE_EINVAL),
    (dict(z_cut=1, kind=W.WAVE_ELASTIC, vs=True), W.WAVE_EINVAL),  # acoustic only
    (dict(precision=7), W.WAVE_EINVAL),
    (dict(precision=W.WAVE_FP16_PAIRS, comp=0), W.WAVE_EINVAL),        # pairs need T
    (dict(precision=W.WAVE_FP16_PAIRS, z_cut=1, n=(16, 16, 16)), W.WAVE_ENOTIMPL),
    (dict(precision=W.WAVE_FP16_PAIRS, kernel=3), W.WAVE_ENOTIMPL),    # one-pass strips
    (dict(kernel=4, n=(16, 16, 16)), W.WAVE_EINVAL),                   # cluster steps are 2D
    (dict(kernel=4, kind=W.WAVE_ELASTIC, vs=True), W.WAVE_EINVAL),     # and acoustic
    (dict(kernel=5), W.WAVE_EINVAL),
])
def test_create_argument_errors(lib, kw, status):
    n = kw.pop("n", (16, 16))
    args = dict(precision=W.WAVE_FP16, comp=3, dt=0.01, spacing=0.1, bc=(1,) * 6,
                field_scale=1.0, kind=W.WAVE_ACOUSTIC)
    rho_scale = kw.pop("rho_scale", 1.0)
    want_vs = kw.pop("vs", False)
    slab = {k: kw.pop(k) for k in ("z_cut", "z0", "kernel") if k in kw}
    args.update(kw)
    with pytest.raises(W.WaveError) as e:
        W.wave_create(n, args["spacing"], _ones(n) * rho_scale, _ones(n), args["dt"],
                      args["precision"], args["comp"], bc=args["bc"], kind=args["kind"],
                      field_scale=args["field_scale"], vs=_ones(n) * 0.5 if want_vs else None, **slab)
    assert e.value.status == status, str(e.value)
    assert W.wave_last_error()


def test_null_context_is_einval(lib):
    import ctypes as C
    assert lib.wave_step(None, 1) == W.WAVE_EINVAL
    assert lib.wave_sync(None) == W.WAVE_EINVAL
    e = C.c_double()
    assert lib.wave_energy(None, C.byref(e)) == W.WAVE_EINVAL
    lib.wave_destroy(None)   # no-op


def test_allocator_pair_required(lib):
    with pytest.raises(W.WaveError):
        W._check(lib.wave_set_allocator(W.ALLOC_FN(lambda n, s, u: None), W.FREE_FN(), None))
    W.use_default_allocator()


def test_static_energy_binding_rejects_bad_tensors(lib):
    """The allocation-free energy entry point takes raw device pointers the
    library cannot check, so the binding checks every tensor first (element
    width of the storage format, element count, layout, output dtype, device)
    and raises before any call into the library."""
    import torch
    n = (16, 12)
    ok16 = torch.zeros(16 * 12, dtype=torch.int16)
    out = torch.zeros(1, dtype=torch.float64)

    def call(prec=W.WAVE_FP16, p=ok16, b=ok16, v=None, o=out, ndim=2):
        v = [ok16, ok16] if v is None else v
        W.wave_energy_acoustic_static(ndim, n, prec, p, p, v, [ok16, ok16], b, 1.0, o)

    cases = [
        (dict(prec=W.WAVE_FP32), "4"),                                 # half arrays for binary32
        (dict(p=torch.zeros(16 * 12, dtype=torch.float32)), "2"),      # binary32 array for half
        (dict(b=torch.zeros(16 * 11, dtype=torch.int16)), "elements"),  # too few points
        (dict(v=[ok16, torch.zeros(24, 16, dtype=torch.int16)[::2]]), "contiguous"),
        (dict(o=torch.zeros(1, dtype=torch.float32)), "float64"),
        (dict(o=torch.zeros(0, dtype=torch.float64)), "float64"),
        (dict(v=[ok16]), "ndim"),
        (dict(ndim=4), "ndim"),
        (dict(), "CUDA"),                                              # everything right but on the host
    ]
    for kw, word in cases:
        with pytest.raises(ValueError) as e:
            call(**kw)
        assert word in str(e.value), (kw, str(e.value))


def test_binding_checks_device_buffers_before_the_call():
    """Receivers, the energy trace, the adjoint residual, the gradient output,
    ghost planes and plane copies take caller device buffers that the library
    cannot check; the binding refuses a tensor of the wrong element type, too
    short, not contiguous, not a tensor, or on the host, before any call into
    the library (the context here has no library object behind it)."""
    import torch
    ctx = W.Context(None, 2, (16, 12, 1), W.WAVE_FP16, W.WAVE_ACOUSTIC)
    recs = [(1, 2), (3, 4), (5, 6)]
    f32 = lambda n: torch.zeros(n, dtype=torch.float32)
    cases = [
        (lambda: W.wave_set_receivers(ctx, W.WAVE_F_P, recs, f32(3 * 10), 10), "CUDA"),
        (lambda: W.wave_set_receivers(ctx, W.WAVE_F_P, recs, f32(3 * 10 - 1), 10), "bytes"),
        (lambda: W.wave_set_receivers(ctx, W.WAVE_F_P, recs, torch.zeros(30, dtype=torch.float64), 10),
         "float32"),
        (lambda: W.wave_set_receivers(ctx, W.WAVE_F_P, recs, f32(60)[::2], 10), "contiguous"),
        (lambda: W.wave_set_receivers(ctx, W.WAVE_F_P, recs, np.zeros(30, np.float32), 10), "torch tensor"),
        (lambda: W.wave_set_energy_trace(ctx, torch.zeros(5, dtype=torch.float64), 6), "bytes"),
        (lambda: W.wave_set_energy_trace(ctx, f32(6), 6), "float64"),
        (lambda: W.wave_set_energy_trace(ctx, torch.zeros(6, dtype=torch.float64), 6), "CUDA"),
        (lambda: W.wave_get_gradient(ctx, f32(16 * 12 - 1)), "bytes"),
        (lambda: W.wave_get_gradient(ctx, torch.zeros(16 * 12, dtype=torch.float16)), "float32"),
        (lambda: W.wave_copy_planes(ctx, W.WAVE_F_P, 0, 2, torch.zeros(64, dtype=torch.int16)), "CUDA"),
        (lambda: W.wave_set_z_ghosts(ctx, None, torch.zeros(64, dtype=torch.int16)), "CUDA"),
    ]
    for call, word in cases:
        with pytest.raises((ValueError, TypeError)) as e:
            call()
        assert word in str(e.value), (word, str(e.value))
    # the residual of a recorded run of 7 steps at 3 receivers
    ctx.nrec, ctx.recorded_steps = 3, 7
    for res, word in [(f32(20), "bytes"), (torch.zeros(21, dtype=torch.float64), "float32"), (f32(21), "CUDA")]:
        with pytest.raises(ValueError) as e:
            W.wave_adjoint_step(ctx, 7, res)
        assert word in str(e.value), (word, str(e.value))
