"""Thin ctypes binding of the C ABI in include/wave.h (same names).

Only argument marshalling lives here: every step of the computation runs in
libwave.so's CUDA kernels. torch supplies the CUDA stream (and, optionally,
device memory through the caching allocator). Loading fails loudly if the
library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwave.so")

WAVE_OK, WAVE_EINVAL, WAVE_ENOMEM, WAVE_ERANGE, WAVE_ECUDA, WAVE_ETIMEOUT, WAVE_ESTATE, \
    WAVE_ENOTIMPL = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ERANGE", "ECUDA", "ETIMEOUT", "ESTATE", "ENOTIMPL"]
WAVE_ACOUSTIC, WAVE_ELASTIC = 0, 1
WAVE_FP64, WAVE_FP32, WAVE_FP16, WAVE_BF16, WAVE_FP16_F32ARITH, WAVE_BF16_F32ARITH, WAVE_FP16_PAIRS = range(7)
WAVE_COMP_NONE, WAVE_COMP_3OP, WAVE_COMP_6OP = 0, 3, 6
WAVE_BC_PERIODIC, WAVE_BC_RIGID, WAVE_BC_FREE = 0, 1, 2
WAVE_F_P, WAVE_F_VX, WAVE_F_VY, WAVE_F_VZ, WAVE_F_SXX, WAVE_F_SYY, WAVE_F_SXY = range(7)

PRECISIONS = {"fp32": WAVE_FP32, "fp16": WAVE_FP16, "bf16": WAVE_BF16,
              "fp16_f32arith": WAVE_FP16_F32ARITH, "bf16_f32arith": WAVE_BF16_F32ARITH,
              "fp16_pairs": WAVE_FP16_PAIRS,
              "fp64": WAVE_FP64}

# Every symbol include/wave.h declares.
EXPORTS = ["wave_set_allocator", "wave_create", "wave_set_initial", "wave_set_source",
           "wave_set_receivers", "wave_step", "wave_set_energy_trace", "wave_energy",
           "wave_get_field", "wave_get_raw", "wave_set_raw", "wave_get_coefficient",
           "wave_get_state", "wave_set_state", "wave_sync", "wave_steps_done",
           "wave_adjoint_step", "wave_destroy", "wave_last_error", "wave_build_info",
           "wave_set_timing", "wave_get_timing", "wave_energy_acoustic_static",
           "wave_batch_create", "wave_batch_step", "wave_batch_set_shape", "wave_batch_info", "wave_batch_destroy",
           "wave_record", "wave_get_gradient", "wave_reset", "wave_selftest_timeout",
           "wave_set_z_ghosts", "wave_half_step", "wave_copy_planes", "wave_get_layout"]


class WaveError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class wave_grid(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("n", C.c_int64 * 3)]


class wave_materials(C.Structure):
    _fields_ = [("kind", C.c_int32), ("rho", C.POINTER(C.c_double)),
                ("vp", C.POINTER(C.c_double)), ("vs", C.POINTER(C.c_double)),
                ("bc", C.c_int32 * 6)]


class wave_options(C.Structure):
    _fields_ = [("field_scale", C.c_double), ("kernel", C.c_int32), ("zchunk", C.c_int32),
                ("z_cut", C.c_int32), ("reserved", C.c_int32 * 5), ("z0", C.c_double),
                ("rho_above", C.POINTER(C.c_double))]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

_lib = None


def lib() -> C.CDLL:
    """Load libwave.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libwave.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dp = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double)
    sig = {
        "wave_set_allocator": [ALLOC_FN, FREE_FN, vp],
        "wave_create": [C.POINTER(wave_grid), dp, C.POINTER(wave_materials), C.c_double, C.c_int,
                        C.c_int, C.POINTER(wave_options), vp, C.POINTER(vp)],
        "wave_set_initial": [vp, C.c_int, dp],
        "wave_set_source": [vp, C.c_int, C.POINTER(C.c_int64), dp, i64],
        "wave_set_receivers": [vp, C.c_int, C.POINTER(C.c_int64), i64, vp, i64],
        "wave_step": [vp, i64],
        "wave_set_energy_trace": [vp, vp, i64],
        "wave_energy": [vp, dp],
        "wave_get_field": [vp, C.c_int, dp],
        "wave_get_raw": [vp, C.c_int, i32, vp],
        "wave_set_raw": [vp, C.c_int, i32, vp],
        "wave_get_coefficient": [vp, i32, dp, dp],
        "wave_get_state": [vp, vp, C.POINTER(C.c_size_t)],
        "wave_set_state": [vp, vp, C.c_size_t],
        "wave_sync": [vp],
        "wave_steps_done": [vp, C.POINTER(C.c_int64)],
        "wave_adjoint_step": [vp, i64, vp],
        "wave_set_timing": [vp, i32],
        "wave_get_timing": [vp, i32, C.POINTER(C.c_int64), dp],
        "wave_energy_acoustic_static": [i32, C.POINTER(C.c_int64), C.c_int, vp, vp,
                                        C.POINTER(vp), C.POINTER(vp), vp, C.c_double, vp, vp],
        "wave_record": [vp, i64, i64],
        "wave_reset": [vp],
        "wave_selftest_timeout": [vp],
        "wave_get_gradient": [vp, vp, C.POINTER(C.c_int64)],
        "wave_batch_create": [i32, C.POINTER(vp), C.POINTER(vp)],
        "wave_batch_step": [vp, i64],
        "wave_batch_set_shape": [vp, i32],
        "wave_batch_info": [vp, C.POINTER(C.c_int32), i32],
        "wave_set_z_ghosts": [vp, vp, vp, vp, vp],
        "wave_half_step": [vp, i32],
        "wave_copy_planes": [vp, C.c_int, i64, i64, vp],
        "wave_get_layout": [vp, C.POINTER(C.c_int64)],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.wave_destroy.argtypes = [vp]
    L.wave_destroy.restype = None
    L.wave_batch_destroy.argtypes = [vp]
    L.wave_batch_destroy.restype = None
    L.wave_last_error.restype = C.c_char_p
    L.wave_build_info.restype = C.c_char_p
    _lib = L
    return L


def wave_last_error() -> str:
    return lib().wave_last_error().decode()


def wave_build_info() -> str:
    return lib().wave_build_info().decode()


def _check(st: int):
    if st != WAVE_OK:
        raise WaveError(st, wave_last_error())


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _torch():
    import torch
    return torch


class Context:
    """Handle returned by wave_create: the opaque pointer plus the grid shape."""

    def __init__(self, ptr, ndim, n, prec, kind):
        self.ptr = ptr
        self.ndim = ndim
        self.n = tuple(n)
        self.prec = prec
        self.kind = kind
        self.nrec = 0           # receivers set (wave_set_receivers)
        self.recorded_steps = 0  # steps of the recorded run (wave_record)

    @property
    def shape(self):
        """numpy shape of one field: (z, y, x) or (y, x)."""
        return tuple(self.n[: self.ndim][::-1])

    @property
    def npts(self):
        return int(np.prod(self.n[: self.ndim]))


def _device_buffer(t, name, min_bytes, dtype=None):
    """Check a caller's device tensor before its pointer goes to the library,
    which cannot check device pointers (a short or misplaced buffer would be
    read or written past its end on the device): a torch tensor of `dtype`
    (any element type when None), at least min_bytes long, contiguous, on a
    CUDA device. Raises TypeError / ValueError."""
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: a torch tensor is required, got {type(t).__name__}")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name}: {t.dtype}, the library writes {dtype}")
    nbytes = t.numel() * t.element_size()
    if nbytes < min_bytes:
        raise ValueError(f"{name}: {nbytes} bytes, the call needs {min_bytes}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: not contiguous")
    if not t.is_cuda:
        raise ValueError(f"{name}: not a CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _stream_handle(stream):
    if stream is not None:
        return stream
    import torch
    if torch.cuda.is_available():
        return torch.cuda.current_stream().cuda_stream
    return None


def wave_create(n, spacing, rho, vp, dt, precision, comp, vs=None, bc=(WAVE_BC_RIGID,) * 6,
                kind=WAVE_ACOUSTIC, field_scale=1.0, kernel=0, zchunk=0, stream=None,
                z_cut=0, z0=0.0, rho_above=None) -> Context:
    """n: cells per axis (x, y[, z]); rho, vp, vs: arrays shaped like a field.
    z_cut, z0, rho_above: a z slab of a larger grid (wave_options in wave.h)."""
    ndim = len(n)
    g = wave_grid()
    g.ndim = ndim
    for ax in range(3):
        g.n[ax] = n[ax] if ax < ndim else 1
    sp = (C.c_double * 3)(*([float(spacing)] * 3 if np.isscalar(spacing) else list(spacing) + [0.0] * (3 - len(spacing))))
    rho_a, rho_p = _f64(rho)
    vp_a, vp_p = _f64(vp)
    m = wave_materials()
    m.kind = kind
    m.rho = rho_p
    m.vp = vp_p
    keep = [rho_a, vp_a]
    if vs is not None:
        vs_a, vs_p = _f64(vs)
        m.vs = vs_p
        keep.append(vs_a)
    for i in range(6):
        m.bc[i] = bc[i] if i < len(bc) else WAVE_BC_PERIODIC
    o = wave_options()
    o.field_scale = field_scale
    o.kernel = kernel
    o.zchunk = zchunk
    o.z_cut = z_cut
    o.z0 = z0
    if rho_above is not None:
        ra, rp = _f64(rho_above)
        keep.append(ra)
        o.rho_above = rp
    out = C.c_void_p()
    _check(lib().wave_create(C.byref(g), sp, C.byref(m), float(dt), int(precision), int(comp),
                             C.byref(o), _stream_handle(stream), C.byref(out)))
    return Context(out, ndim, [g.n[0], g.n[1], g.n[2]], precision, kind)


def wave_destroy(ctx: Context):
    if ctx.ptr:
        lib().wave_destroy(ctx.ptr)
        ctx.ptr = None


def wave_set_initial(ctx: Context, field: int, values):
    a, p = _f64(values)
    assert a.size == ctx.npts
    _check(lib().wave_set_initial(ctx.ptr, field, p))


def wave_set_source(ctx: Context, field: int, idx, wavelet):
    ix = (C.c_int64 * 3)(*(list(idx) + [0] * (3 - len(idx))))
    w, wp = _f64(wavelet)
    _check(lib().wave_set_source(ctx.ptr, field, ix, wp, w.size))


def wave_set_receivers(ctx: Context, field: int, idx, traces=None, capacity_steps=0):
    """idx: sequence of (i, j[, k]); traces: float32 CUDA tensor of at least
    capacity_steps * nrec elements (checked here)."""
    idx = np.asarray(idx, dtype=np.int64).reshape(len(idx), -1) if len(idx) else np.zeros((0, 3), np.int64)
    full = np.zeros((idx.shape[0], 3), np.int64)
    full[:, : idx.shape[1]] = idx
    full = np.ascontiguousarray(full)
    ptr = None
    if traces is not None:
        need = 4 * max(int(capacity_steps), 0) * full.shape[0]
        ptr = _device_buffer(traces, "traces", need, _torch().float32)
    _check(lib().wave_set_receivers(ctx.ptr, field, full.ctypes.data_as(C.POINTER(C.c_int64)),
                                    full.shape[0], ptr, capacity_steps))
    ctx.nrec = full.shape[0]


def wave_step(ctx: Context, n: int):
    _check(lib().wave_step(ctx.ptr, int(n)))


def wave_half_step(ctx: Context, which: int):
    _check(lib().wave_half_step(ctx.ptr, int(which)))


def wave_set_z_ghosts(ctx: Context, p_lo=None, p_hi=None, vz_lo=None, vz_hi=None):
    """Ghost-plane buffers (CUDA tensors of at least two planes each, laid out
    as wave_get_layout says; checked here) of the cut faces; None for a face
    of the grid."""
    bufs = list(zip(("p_lo", "p_hi", "vz_lo", "vz_hi"), (p_lo, p_hi, vz_lo, vz_hi)))
    for nm, t in bufs:
        if t is not None:
            _device_buffer(t, nm, 0)
    need = 0
    if any(t is not None for _, t in bufs):
        _, plane, eb = wave_get_layout(ctx)
        need = 2 * plane * eb
    ptrs = [None if t is None else _device_buffer(t, nm, need) for nm, t in bufs]
    _check(lib().wave_set_z_ghosts(ctx.ptr, *ptrs))


def wave_copy_planes(ctx: Context, field: int, z_first: int, nplanes: int, dst):
    """Copy planes z_first .. z_first + nplanes - 1 of a field into the CUDA
    tensor dst (at least nplanes planes of the layout; checked here)."""
    _device_buffer(dst, "dst", 0)
    _, plane, eb = wave_get_layout(ctx)
    ptr = _device_buffer(dst, "dst", max(int(nplanes), 0) * plane * eb)
    _check(lib().wave_copy_planes(ctx.ptr, field, int(z_first), int(nplanes), ptr))


def wave_get_layout(ctx: Context):
    """(row pitch in elements, elements per plane, bytes per element)."""
    out = (C.c_int64 * 3)()
    _check(lib().wave_get_layout(ctx.ptr, out))
    return int(out[0]), int(out[1]), int(out[2])


def wave_set_energy_trace(ctx: Context, device_energy=None, capacity=0):
    """device_energy: float64 CUDA tensor of at least capacity elements (checked here)."""
    ptr = None
    if device_energy is not None:
        ptr = _device_buffer(device_energy, "device_energy", 8 * max(int(capacity), 0), _torch().float64)
    _check(lib().wave_set_energy_trace(ctx.ptr, ptr, capacity))


def wave_energy(ctx: Context) -> float:
    e = C.c_double()
    _check(lib().wave_energy(ctx.ptr, C.byref(e)))
    return e.value


def wave_get_field(ctx: Context, field: int) -> np.ndarray:
    out = np.empty(ctx.shape, np.float64)
    _check(lib().wave_get_field(ctx.ptr, field, out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def _raw_dtype(prec):
    return np.float32 if prec == WAVE_FP32 else np.uint16


def wave_get_raw(ctx: Context, field: int, compensation: int = 0) -> np.ndarray:
    out = np.empty(ctx.shape, _raw_dtype(ctx.prec))
    _check(lib().wave_get_raw(ctx.ptr, field, compensation, out.ctypes.data_as(C.c_void_p)))
    return out


def wave_set_raw(ctx: Context, field: int, compensation: int, values):
    a = np.ascontiguousarray(values, dtype=_raw_dtype(ctx.prec))
    _check(lib().wave_set_raw(ctx.ptr, field, compensation, a.ctypes.data_as(C.c_void_p)))


def wave_get_coefficient(ctx: Context, which: int):
    out = np.empty(ctx.shape, np.float64)
    z0 = C.c_double()
    _check(lib().wave_get_coefficient(ctx.ptr, which, out.ctypes.data_as(C.POINTER(C.c_double)),
                                      C.byref(z0)))
    return out, z0.value


def wave_get_state(ctx: Context) -> bytes:
    size = C.c_size_t(0)
    _check(lib().wave_get_state(ctx.ptr, None, C.byref(size)))
    buf = C.create_string_buffer(size.value)
    _check(lib().wave_get_state(ctx.ptr, buf, C.byref(size)))
    return buf.raw[: size.value]


def wave_set_state(ctx: Context, blob: bytes):
    buf = C.create_string_buffer(blob, len(blob))
    _check(lib().wave_set_state(ctx.ptr, buf, len(blob)))


def wave_sync(ctx: Context):
    _check(lib().wave_sync(ctx.ptr))


def wave_steps_done(ctx: Context) -> int:
    s = C.c_int64()
    _check(lib().wave_steps_done(ctx.ptr, C.byref(s)))
    return s.value


def wave_selftest_timeout(ctx: Context):
    """Force a bounded device wait to expire; raises WaveError(ETIMEOUT)."""
    _check(lib().wave_selftest_timeout(ctx.ptr))


def wave_reset(ctx: Context):
    """Zero the fields, compensations and step counter (keeps medium, source, receivers)."""
    _check(lib().wave_reset(ctx.ptr))


def wave_record(ctx: Context, nsteps: int, ncheckpoints: int = 0):
    """Forward run of nsteps steps with checkpoints for the adjoint."""
    _check(lib().wave_record(ctx.ptr, int(nsteps), int(ncheckpoints)))
    ctx.recorded_steps = int(nsteps)


def wave_adjoint_step(ctx: Context, n: int, residual=None):
    """n adjoint steps; residual: float32 CUDA tensor [nsteps, nrec] of the
    recorded run (its size is checked here)."""
    ptr = None
    if residual is not None:
        need = 4 * ctx.recorded_steps * ctx.nrec
        ptr = _device_buffer(residual, "residual", need, _torch().float32)
    _check(lib().wave_adjoint_step(ctx.ptr, int(n), ptr))


def wave_get_gradient(ctx: Context, out=None):
    """dJ/dc as a float32 CUDA tensor shaped like the fields ((z,) y, x);
    returns (gradient, adjoint steps left)."""
    torch = _torch()
    if out is None:
        out = torch.empty(tuple(ctx.n[:ctx.ndim][::-1]), dtype=torch.float32, device="cuda")
    ptr = _device_buffer(out, "out", 4 * ctx.npts, torch.float32)
    left = C.c_int64()
    _check(lib().wave_get_gradient(ctx.ptr, ptr, C.byref(left)))
    return out, left.value


def wave_set_timing(ctx: Context, enable: bool):
    _check(lib().wave_set_timing(ctx.ptr, 1 if enable else 0))


def wave_get_timing(ctx: Context, kind: int):
    """(launches, total milliseconds) for kernel kind 0 velocity, 1 pressure, 2 receivers."""
    n = C.c_int64()
    ms = C.c_double()
    _check(lib().wave_get_timing(ctx.ptr, kind, C.byref(n), C.byref(ms)))
    return n.value, ms.value


def wave_energy_acoustic_static(ndim, n, precision, p_old, p_new, v, a, b, factor, device_out,
                                stream=None):
    """The acoustic discrete energy from device tensors the caller owns, with
    no device allocation inside the library (for callers that cannot call
    cudaMalloc, such as a framework that reserves the whole device heap, or a
    loop whose memory budget forbids allocating after start-up). All array
    arguments are contiguous torch CUDA tensors in the storage format (2-byte
    elements for the half and bfloat16 codes, 4-byte for WAVE_FP32) with at
    least prod(n[:ndim]) elements; device_out is a float64 CUDA tensor of at
    least one element. The library cannot check device pointers, so this
    binding checks the tensors and raises ValueError before the call."""
    if ndim not in (2, 3) or len(n) < ndim or len(v) != ndim or len(a) != ndim:
        raise ValueError("ndim must be 2 or 3, with ndim extents, velocities and multipliers")
    npts = 1
    for d in range(ndim):
        if int(n[d]) < 1:
            raise ValueError(f"n[{d}] must be positive")
        npts *= int(n[d])
    width = 4 if int(precision) == WAVE_FP32 else 2
    named = [("p_old", p_old), ("p_new", p_new), ("b", b)]
    named += [(f"v[{d}]", t) for d, t in enumerate(v)] + [(f"a[{d}]", t) for d, t in enumerate(a)]
    for name, t in named:
        if t.element_size() != width:
            raise ValueError(f"{name}: {t.element_size()}-byte elements, the storage format has {width}")
        if t.numel() < npts:
            raise ValueError(f"{name}: {t.numel()} elements, the grid has {npts}")
        if not t.is_contiguous():
            raise ValueError(f"{name}: not contiguous")
    import torch
    if device_out.dtype != torch.float64 or device_out.numel() < 1:
        raise ValueError("device_out must be a float64 tensor of at least one element")
    for name, t in named + [("device_out", device_out)]:
        if not t.is_cuda:
            raise ValueError(f"{name}: not a CUDA tensor")
    nn = (C.c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
    vv = (C.c_void_p * 3)(*([t.data_ptr() for t in v] + [None] * (3 - len(v))))
    aa = (C.c_void_p * 3)(*([t.data_ptr() for t in a] + [None] * (3 - len(a))))
    _check(lib().wave_energy_acoustic_static(
        ndim, nn, int(precision), C.c_void_p(p_old.data_ptr()), C.c_void_p(p_new.data_ptr()),
        vv, aa, C.c_void_p(b.data_ptr()), float(factor), C.c_void_p(device_out.data_ptr()),
        _stream_handle(stream)))


class Batch:
    """Handle of wave_batch_create: the opaque pointer and the contexts."""

    def __init__(self, ptr, ctxs):
        self.ptr = ptr
        self.ctxs = list(ctxs)


def wave_batch_create(ctxs) -> Batch:
    arr = (C.c_void_p * len(ctxs))(*[c.ptr for c in ctxs])
    out = C.c_void_p()
    _check(lib().wave_batch_create(len(ctxs), arr, C.byref(out)))
    return Batch(out, ctxs)


def wave_batch_step(batch: Batch, n: int):
    _check(lib().wave_batch_step(batch.ptr, int(n)))


def wave_batch_info(batch: Batch) -> dict:
    """The launch configuration in use (kind, tile, threads, blocks, graph
    steps, tuned)."""
    v = (C.c_int32 * 7)()
    _check(lib().wave_batch_info(batch.ptr, v, 7))
    return {"kind": ("points", "strips", "one-pass strips", "persistent strips")[v[0]], "tile_x": v[1], "tile_y": v[2], "threads": v[3],
            "blocks": v[4], "graph_steps": v[5], "tuned": bool(v[6])}


def wave_batch_set_shape(batch: Batch, shape: int):
    """Use candidate launch shape `shape` of the tuner's list instead of tuning
    (0-1 tiles of points, 2-13 two-launch strips, 14-17 persistent strips,
    18-23 one-pass strips)."""
    _check(lib().wave_batch_set_shape(batch.ptr, int(shape)))


def wave_batch_destroy(batch: Batch):
    if batch.ptr:
        lib().wave_batch_destroy(batch.ptr)
        batch.ptr = None


# ---------------------------------------------------------------- allocator
_alloc_cbs = None


def use_torch_allocator(device: int = 0):
    """Route the library's device allocations through torch's caching allocator."""
    import torch
    global _alloc_cbs

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream or 0)
        except Exception:
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    _alloc_cbs = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(lib().wave_set_allocator(_alloc_cbs[0], _alloc_cbs[1], None))


def use_default_allocator():
    global _alloc_cbs
    _check(lib().wave_set_allocator(ALLOC_FN(), FREE_FN(), None))
    _alloc_cbs = None
