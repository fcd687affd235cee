"""CPU oracle for the half-precision staggered-grid wave scheme -- TEST INFRASTRUCTURE.

This package is the reference that the CUDA path is checked against. It is a
plain, slow restatement of Gao & Harms, "Half precision wave simulation"
(arXiv 2310.00236): the fourth-order staggered leapfrog scheme of Section 3
(Eq. 1 acoustic, Eq. 2 elastic in Appendix A) with every operation rounded to
a chosen format, and the plain (Algorithm 1) or compensated (Algorithm 2,
Code 1 / Code 2) solution update.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it. It shares no code with the CUDA path and never
imports the product package.

Parity status of each function is stated in its docstring; functions without a
pin that is independent of this file say "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wave_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

FP64, FP32, FP16, BF16 = 0, 1, 2, 3
BC_PERIODIC, BC_RIGID = 0, 1
FORMAT_NAMES = {"fp64": FP64, "fp32": FP32, "fp16": FP16, "bf16": BF16}


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc, no contraction, no fast-math, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-fopenmp", _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        i64 = C.c_int64
        L.orc_round.restype = C.c_double
        L.orc_round.argtypes = [C.c_double, C.c_int]
        L.orc_round_array.argtypes = [i64, dp, C.c_int, dp]
        L.orc_op_array.argtypes = [i64, C.c_int, dp, dp, C.c_int, dp]
        L.orc_sum_op_array.argtypes = [i64, C.c_int, dp, dp, C.c_int, dp, dp]
        L.orc_update_array.argtypes = [i64, C.c_int, C.c_int, C.c_int, dp, dp, dp, dp, dp]
        L.orc_stencil_c2.restype = C.c_double
        L.orc_stencil_c2.argtypes = [C.c_int]
        L.orc_set_threads.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_acoustic_apply_walls.argtypes = [C.c_void_p, dp, dp, dp, dp]
        L.orc_acoustic_run.restype = C.c_int
        L.orc_acoustic_run.argtypes = ([C.c_void_p] + [dp] * 8 + [dp] * 4 +
                                       [i64, i64, i64, i64, dp, C.c_int32, i64,
                                        C.POINTER(C.c_int64), dp, dp])
        L.orc_acoustic_adjoint.restype = C.c_int
        L.orc_acoustic_adjoint.argtypes = ([C.c_void_p] + [dp] * 4 + [dp] * 4 + [dp] +
                                           [i64, i64, i64, i64, dp, i64, C.POINTER(C.c_int64),
                                            dp, dp, dp, dp, dp])
        L.orc_acoustic_coefficients.restype = C.c_int
        L.orc_acoustic_coefficients.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double,
                                                dp, dp, dp, dp, dp, dp, dp]
        L.orc_scale_pressure.argtypes = [i64, dp, C.c_double, C.c_int, dp]
        L.orc_scale_velocity.argtypes = [i64, dp, C.c_double, C.c_double, C.c_int, dp]
        L.orc_scale_source.argtypes = [i64, dp, C.c_double, C.c_double, C.c_double, C.c_int,
                                       C.c_int, dp]
        L.orc_acoustic_half_step.restype = C.c_int
        L.orc_acoustic_half_step.argtypes = ([C.c_void_p, C.c_int32] + [dp] * 8 + [dp] * 4 + [dp, dp] +
                                             [i64, i64, i64, dp])
        L.orc_energy_factor.restype = C.c_double
        L.orc_energy_factor.argtypes = [C.c_double] * 4 + [C.c_int]
        _lib = L
    return _lib


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Formats and arithmetic (Section 2, Table 1)
# --------------------------------------------------------------------------

def round_to(x, fmt: int) -> np.ndarray:
    """Round binary64 values to the nearest value of `fmt`, ties to even.

    Pinned against numpy's binary16 / binary32 conversions and torch's
    bfloat16 conversion, and against the Table 1 constants.
    """
    x = _f64(x)
    out = np.empty_like(x)
    lib().orc_round_array(x.size, _dp(x), fmt, _dp(out))
    return out


def op(name: str, a, b, fmt: int) -> np.ndarray:
    """Correctly rounded a+b, a-b or a*b in `fmt` (Section 2's IEEE model).

    Pinned against numpy float16/float32 and torch bfloat16 arithmetic.
    """
    a, b = np.broadcast_arrays(_f64(a), _f64(b))
    a, b = _f64(a), _f64(b)
    out = np.empty_like(a)
    lib().orc_op_array(a.size, {"add": 0, "sub": 1, "mul": 2}[name], _dp(a), _dp(b), fmt, _dp(out))
    return out


def compensated_sum(variant: int, a, b, fmt: int):
    """sum_3op (Code 1) or sum_6op (Code 2) of Section 4, element-wise.

    Pinned by the error-free-transformation identity a + b = s + t checked in
    exact (binary64) arithmetic, for sum_3op when |a| >= |b|.
    """
    a, b = np.broadcast_arrays(_f64(a), _f64(b))
    a, b = _f64(a), _f64(b)
    s = np.empty_like(a)
    t = np.empty_like(a)
    lib().orc_sum_op_array(a.size, variant, _dp(a), _dp(b), fmt, _dp(s), _dp(t))
    return s, t


def solution_update(comp: int, V, T, inc, store_fmt: int, arith_fmt: int):
    """The solution update of Algorithms 1 / 2 as the solvers apply it,
    element-wise: V += inc (comp = 0), or R = T + inc and the compensated sum
    of (V, R) giving the new (V, T) (comp = 3 or 6). With a wider arithmetic
    format than the storage format (reading A5: half storage, binary32
    registers), s = V + R in the arithmetic format, V' = RN(s), T' = RN(s - V').
    Returns (V', T').

    Pinned in tests/test_oracle_eft.py by properties computed with numpy's own
    binary16 / binary32 arithmetic (the pair (V', T') represents
    V + (T + inc) within the rounding of T'; a dropped, negated or unrounded
    T fails them).
    """
    V, T, inc = np.broadcast_arrays(_f64(V), _f64(T), _f64(inc))
    V, T, inc = _f64(V), _f64(T), _f64(inc)
    Vo = np.empty_like(V)
    To = np.empty_like(V)
    lib().orc_update_array(V.size, comp, arith_fmt, store_fmt, _dp(V), _dp(T), _dp(inc),
                           _dp(Vo), _dp(To))
    return Vo, To


def stencil_c2(fmt: int) -> float:
    """The 1/24 stencil weight rounded to `fmt` (Section 3)."""
    return lib().orc_stencil_c2(fmt)


# --------------------------------------------------------------------------
# Acoustic solver (Eq. 1, Algorithms 1 and 2)
# --------------------------------------------------------------------------

def set_threads(n: int = 0) -> int:
    """Set the OpenMP thread count of the solvers (n <= 0 leaves it) and return
    the count in force. The results do not depend on it: every parallel loop
    writes disjoint points and the energy partial sums are combined in a fixed
    order (pinned by the thread-count invariance test)."""
    return int(lib().orc_set_threads(int(n)))


class AcousticCfg(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("bc", C.c_int32 * 3), ("n", C.c_int64 * 3),
                ("store_fmt", C.c_int32), ("arith_fmt", C.c_int32),
                ("stencil_fmt", C.c_int32), ("comp", C.c_int32), ("c2_override", C.c_int32),
                ("pair_stencil", C.c_int32)]


def acoustic_cfg(shape, bc, store_fmt, comp, arith_fmt=None, stencil_fmt=None,
                 c2_fmt=None, pair_stencil=False) -> AcousticCfg:
    """shape: cells per axis, ordered (x, y[, z]); bc: one code per axis.
    c2_fmt: round the stencil weight 1/24 to this format instead of the
    stencil format (an experiment on the operator's rounding; None: the
    scheme). pair_stencil: the stencils read RN(V + T), the stored value plus
    its compensation, instead of V (an experiment, not the paper's scheme)."""
    nd = len(shape)
    cfg = AcousticCfg()
    cfg.ndim = nd
    for ax in range(3):
        cfg.n[ax] = shape[ax] if ax < nd else 1
        cfg.bc[ax] = bc[ax] if ax < nd else BC_PERIODIC
    cfg.store_fmt = store_fmt
    cfg.arith_fmt = store_fmt if arith_fmt is None else arith_fmt
    cfg.stencil_fmt = cfg.arith_fmt if stencil_fmt is None else stencil_fmt
    cfg.comp = comp
    cfg.c2_override = 0 if c2_fmt is None else 1 + c2_fmt
    cfg.pair_stencil = 1 if pair_stencil else 0
    return cfg


class AcousticState:
    """Fields stored as numpy float64 arrays shaped (z, y, x) (or (y, x) in 2D),
    x fastest, each value representable in the storage format."""

    def __init__(self, cfg: AcousticCfg):
        self.cfg = cfg
        nd = cfg.ndim
        self.shape = tuple(int(cfg.n[a]) for a in range(nd))[::-1]
        z = lambda: np.zeros(self.shape, np.float64)
        self.p, self.tp = z(), z()
        self.v = [z() for _ in range(3)]
        self.tv = [z() for _ in range(3)]
        self.a = [np.zeros(self.shape) for _ in range(3)]
        self.b = np.zeros(self.shape)
        self.step = 0
        self.src_index = -1
        self.src = None

    def copy(self):
        s = AcousticState(self.cfg)
        s.p, s.tp = self.p.copy(), self.tp.copy()
        s.v = [x.copy() for x in self.v]
        s.tv = [x.copy() for x in self.tv]
        s.a = [x.copy() for x in self.a]
        s.b = self.b.copy()
        s.step, s.src_index, s.src = self.step, self.src_index, self.src
        return s

    def apply_walls(self):
        lib().orc_acoustic_apply_walls(C.byref(self.cfg), _dp(self.p), _dp(self.v[0]),
                                       _dp(self.v[1]), _dp(self.v[2]))

    def run(self, nsteps: int, rec_field: int = 0, rec_index=None, energy: bool = False):
        """Advance `nsteps` steps; returns (traces [nsteps, nrec] or None,
        scaled energies [nsteps] or None)."""
        nrec = 0 if rec_index is None else len(rec_index)
        traces = np.zeros((nsteps, nrec)) if nrec else None
        en = np.zeros(nsteps) if energy else None
        ri = None
        if nrec:
            ri_arr = np.ascontiguousarray(rec_index, dtype=np.int64)
            ri = ri_arr.ctypes.data_as(C.POINTER(C.c_int64))
        src = None if self.src is None else _f64(self.src)
        rc = lib().orc_acoustic_run(
            C.byref(self.cfg), _dp(self.p), _dp(self.tp), _dp(self.v[0]), _dp(self.tv[0]),
            _dp(self.v[1]), _dp(self.tv[1]), _dp(self.v[2]), _dp(self.tv[2]),
            _dp(self.a[0]), _dp(self.a[1]), _dp(self.a[2]), _dp(self.b),
            nsteps, self.step, self.src_index, 0 if src is None else src.size, _dp(src),
            rec_field, nrec, ri, _dp(traces), _dp(en))
        if rc != 0:
            raise MemoryError("oracle run failed")
        self.step += nsteps
        return traces, en


def acoustic_half_step(st: AcousticState, which: int, ghost_lo=None, ghost_hi=None):
    """One half step of a 3D z slab (domain decomposition along z; not in the
    paper): which = 0 velocities from p, 1 pressure from the velocities (at
    global step st.step, which then advances), with the same operations as
    AcousticState.run. ghost_lo / ghost_hi: the grid planes z0-2, z0-1 and
    z1, z1+1 of the field the half step differentiates along z (p, then v_z),
    arrays shaped (2, ny, nx); None where the slab's face is a face of the
    grid. Pinned by tests/test_zslab_cpu.py: slabs stepped with exchanged
    ghosts reproduce the whole grid's run bit for bit."""
    lo = None if ghost_lo is None else _f64(ghost_lo)
    hi = None if ghost_hi is None else _f64(ghost_hi)
    src = None if st.src is None else _f64(st.src)
    rc = lib().orc_acoustic_half_step(
        C.byref(st.cfg), int(which), _dp(st.p), _dp(st.tp), _dp(st.v[0]), _dp(st.tv[0]), _dp(st.v[1]),
        _dp(st.tv[1]), _dp(st.v[2]), _dp(st.tv[2]), _dp(st.a[0]), _dp(st.a[1]), _dp(st.a[2]), _dp(st.b),
        _dp(lo), _dp(hi), st.step, st.src_index, 0 if src is None else src.size, _dp(src))
    if rc != 0:
        raise ValueError("the slab half step takes 3D states without pair_stencil")
    if which == 1:
        st.step += 1


def acoustic_adjoint(st: AcousticState, c, nsteps: int, rec_index, residual=None, d_obs=None):
    """Discrete adjoint (reverse mode) of `nsteps` binary64 steps from the
    state `st` (not modified), for the pressure traces at rec_index.

    J = 1/2 sum (trace - d_obs)^2 when d_obs is given (residual = trace -
    d_obs), else the adjoint of the linear functional sum residual * trace.
    c: the velocity model the coefficients b were made from.
    Returns dict(traces, J, grad_b, grad_c, p0_bar). The state must be binary64
    without compensation.

    Pinned by tests/test_oracle_adjoint.py: the dot-product identity
    <F x, y> = <x, F^T y> of the linear map from the initial pressure to the
    traces, and central finite differences of the forward misfit in c.
    """
    ri = np.ascontiguousarray(rec_index, dtype=np.int64)
    nrec = ri.size
    if d_obs is not None:
        tr, _ = st.copy().run(nsteps, 0, ri)
        residual = tr - np.asarray(d_obs, dtype=np.float64).reshape(nsteps, nrec)
    res = _f64(np.asarray(residual, dtype=np.float64).reshape(nsteps, nrec))
    traces = np.zeros((nsteps, nrec))
    gb, gc, p0b = np.zeros(st.shape), np.zeros(st.shape), np.zeros(st.shape)
    src = None if st.src is None else _f64(st.src)
    rc = lib().orc_acoustic_adjoint(
        C.byref(st.cfg), _dp(_f64(st.p)), _dp(_f64(st.v[0])), _dp(_f64(st.v[1])), _dp(_f64(st.v[2])),
        _dp(st.a[0]), _dp(st.a[1]), _dp(st.a[2]), _dp(st.b), _dp(_f64(c).reshape(st.shape)), nsteps,
        st.step, st.src_index, 0 if src is None else src.size, _dp(src), nrec,
        ri.ctypes.data_as(C.POINTER(C.c_int64)), _dp(res), _dp(traces), _dp(gb), _dp(gc), _dp(p0b))
    if rc == -2:
        raise ValueError("the adjoint oracle takes binary64 states without compensation")
    if rc != 0:
        raise MemoryError("oracle adjoint failed")
    J = None if d_obs is None else 0.5 * float(np.sum(res * res))
    return {"traces": traces, "J": J, "grad_b": gb, "grad_c": gc, "p0_bar": p0b}


def acoustic_coefficients(cfg: AcousticCfg, h: float, dt: float, P0: float, rho, c):
    """Per-point multipliers a_x, a_y, a_z (at v points) and b (at p nodes).

    Returns (a list, b, Z0, ok). Pinned through the uniform case (a = b = CFL,
    exactly) and the exact energy conservation that uses these values.
    """
    rho, c = _f64(rho), _f64(c)
    shape = rho.shape
    a = [np.zeros(shape) for _ in range(3)]
    b = np.zeros(shape)
    z0 = C.c_double(0.0)
    bad = lib().orc_acoustic_coefficients(C.byref(cfg), h, dt, P0, _dp(rho), _dp(c), _dp(a[0]),
                                          _dp(a[1]), _dp(a[2]), _dp(b), C.byref(z0))
    return a, b, z0.value, bad == 0


def scale_pressure(p, P0, fmt):
    """p^ = RN(p / P0) (Section 3's scaled pressure). Pinned by the rounding
    pins and by the physical-units standing mode (a wrong P0 changes the
    physical solution read back as P0 p^)."""
    p = _f64(p)
    out = np.empty_like(p)
    lib().orc_scale_pressure(p.size, _dp(p), P0, fmt, _dp(out))
    return out


def scale_velocity(v, Z0, P0, fmt):
    """v^ = RN(v * Z0 / P0) (Section 3's scaled velocity). Pinned by the
    rounding pins and by the physical-units standing mode with rho, c, P0 far
    from 1 (a wrong or missing Z0 or P0 fails it)."""
    v = _f64(v)
    out = np.empty_like(v)
    lib().orc_scale_velocity(v.size, _dp(v), Z0, P0, fmt, _dp(out))
    return out


def scale_source(w, Z0, P0, h, ndim, fmt):
    """Scaled point-source values s^ = RN(w Z0 / (P0 h^(d-1)))."""
    w = _f64(w)
    out = np.empty_like(w)
    lib().orc_scale_source(w.size, _dp(w), Z0, P0, h, ndim, fmt, _dp(out))
    return out


def energy_factor(h, dt, P0, Z0, ndim) -> float:
    return lib().orc_energy_factor(h, dt, P0, Z0, ndim)


def acoustic_setup(shape, bc, h, dt, rho, c, store_fmt, comp, P0=1.0, arith_fmt=None,
                   stencil_fmt=None, p0=None, v0=None, c2_fmt=None, coef_fmt=None,
                   pair_stencil=False):
    """Build a ready-to-run AcousticState from physical inputs: coefficients
    (rounded once), scaled and rounded initial fields, walls applied.
    c2_fmt / coef_fmt: round the stencil weight 1/24 / the multipliers a and b
    to these formats instead of the scheme's (experiments that separate the
    operator's rounding from the rest; None: the scheme); pair_stencil: see
    acoustic_cfg."""
    cfg = acoustic_cfg(shape, bc, store_fmt, comp, arith_fmt, stencil_fmt, c2_fmt, pair_stencil)
    st = AcousticState(cfg)
    ccfg = cfg if coef_fmt is None else acoustic_cfg(shape, bc, coef_fmt, comp)
    a, b, Z0, ok = acoustic_coefficients(ccfg, h, dt, P0, rho, c)
    if not ok:
        raise ValueError("coefficient outside the storage format's normal range")
    st.a, st.b, st.Z0, st.P0, st.h, st.dt = a, b, Z0, P0, h, dt
    if p0 is not None:
        st.p = scale_pressure(p0, P0, store_fmt).reshape(st.shape)
    if v0 is not None:
        for ax, vv in enumerate(v0):
            if vv is not None:
                st.v[ax] = scale_velocity(vv, Z0, P0, store_fmt).reshape(st.shape)
    st.apply_walls()
    return st


# --------------------------------------------------------------------------
# Elastic solver (Eq. 2, Appendix A)
# --------------------------------------------------------------------------
EBC_PERIODIC, EBC_RIGID, EBC_FREE = 0, 1, 2
# not a physical face: fields read zero beyond it (sub-boxes over a domain of dependence)
EBC_ZERO = 3


class ElasticCfg(C.Structure):
    _fields_ = [("n", C.c_int64 * 2), ("bc", C.c_int32 * 4), ("store_fmt", C.c_int32),
                ("arith_fmt", C.c_int32), ("stencil_fmt", C.c_int32), ("comp", C.c_int32),
                ("pair_stencil", C.c_int32)]


def elastic_cfg(shape, bc, store_fmt, comp, arith_fmt=None, stencil_fmt=None,
                pair_stencil=False) -> ElasticCfg:
    """shape (nx, ny); bc per face (x-lo, x-hi, y-lo, y-hi). pair_stencil: the
    stencils read RN(V + T) (with compensation; not the paper's scheme)."""
    cfg = ElasticCfg()
    cfg.n[0], cfg.n[1] = shape
    for i in range(4):
        cfg.bc[i] = bc[i]
    cfg.store_fmt = store_fmt
    cfg.arith_fmt = store_fmt if arith_fmt is None else arith_fmt
    cfg.stencil_fmt = cfg.arith_fmt if stencil_fmt is None else stencil_fmt
    cfg.comp = comp
    cfg.pair_stencil = 1 if pair_stencil else 0
    return cfg


ELASTIC_FIELDS = ("vx", "vy", "sxx", "syy", "sxy")


class ElasticState:
    """Fields as float64 arrays shaped (ny, nx); f[name] values, t[name] compensations."""

    def __init__(self, cfg: ElasticCfg):
        self.cfg = cfg
        self.shape = (int(cfg.n[1]), int(cfg.n[0]))
        self.f = {k: np.zeros(self.shape) for k in ELASTIC_FIELDS}
        self.t = {k: np.zeros(self.shape) for k in ELASTIC_FIELDS}
        self.coef = {k: np.zeros(self.shape) for k in ("bx", "by", "l2m", "lam", "mu")}
        self.step = 0
        self.src_index = -1
        self.src = None

    def apply_walls(self):
        _elib().orc_elastic_apply_walls(C.byref(self.cfg), _dp(self.f["vx"]), _dp(self.f["vy"]),
                                        _dp(self.f["syy"]), _dp(self.f["sxy"]))

    def run(self, nsteps, rec_field=2, rec_index=None, energy=False):
        nrec = 0 if rec_index is None else len(rec_index)
        traces = np.zeros((nsteps, nrec)) if nrec else None
        en = np.zeros(nsteps) if energy else None
        ri = None
        if nrec:
            ri_arr = np.ascontiguousarray(rec_index, dtype=np.int64)
            ri = ri_arr.ctypes.data_as(C.POINTER(C.c_int64))
        src = None if self.src is None else _f64(self.src)
        f, t, c = self.f, self.t, self.coef
        rc = _elib().orc_elastic_run(
            C.byref(self.cfg), _dp(f["vx"]), _dp(t["vx"]), _dp(f["vy"]), _dp(t["vy"]),
            _dp(f["sxx"]), _dp(t["sxx"]), _dp(f["syy"]), _dp(t["syy"]), _dp(f["sxy"]),
            _dp(t["sxy"]), _dp(c["bx"]), _dp(c["by"]), _dp(c["l2m"]), _dp(c["lam"]), _dp(c["mu"]),
            nsteps, self.step, self.src_index, 0 if src is None else src.size, _dp(src),
            rec_field, nrec, ri, _dp(traces), _dp(en))
        if rc != 0:
            raise MemoryError("oracle run failed")
        self.step += nsteps
        return traces, en


_elib_done = False


def _elib():
    global _elib_done
    L = lib()
    if not _elib_done:
        dp = C.POINTER(C.c_double)
        i64 = C.c_int64
        L.orc_elastic_apply_walls.argtypes = [C.c_void_p, dp, dp, dp, dp]
        L.orc_elastic_run.restype = C.c_int
        L.orc_elastic_run.argtypes = ([C.c_void_p] + [dp] * 10 + [dp] * 5 +
                                      [i64, i64, i64, i64, dp, C.c_int32, i64,
                                       C.POINTER(C.c_int64), dp, dp])
        L.orc_elastic_coefficients.restype = C.c_int
        L.orc_elastic_coefficients.argtypes = [C.c_void_p, C.c_double, C.c_double, dp, dp, dp,
                                               dp, dp, dp, dp, dp, dp]
        L.orc_elastic_scale_source.argtypes = [i64, dp, C.c_double, C.c_double, C.c_double,
                                               C.c_double, C.c_int, dp]
        _elib_done = True
    return L


def elastic_coefficients(cfg: ElasticCfg, h, dt, rho, vp, vs):
    """Multipliers bx, by (velocities), l2m, lam (normal stresses), mu (shear).
    Returns (dict, Z0, ok)."""
    rho, vp, vs = _f64(rho), _f64(vp), _f64(vs)
    out = {k: np.zeros(rho.shape) for k in ("bx", "by", "l2m", "lam", "mu")}
    z0 = C.c_double()
    bad = _elib().orc_elastic_coefficients(C.byref(cfg), h, dt, _dp(rho), _dp(vp), _dp(vs),
                                           _dp(out["bx"]), _dp(out["by"]), _dp(out["l2m"]),
                                           _dp(out["lam"]), _dp(out["mu"]), C.byref(z0))
    return out, z0.value, bad == 0


def elastic_scale_source(w, dt, Z0, P0, h, fmt):
    """v_y source in increment units s^ = RN(w dt Z0 / (P0 h^2))."""
    w = _f64(w)
    out = np.empty_like(w)
    _elib().orc_elastic_scale_source(w.size, _dp(w), dt, Z0, P0, h, fmt, _dp(out))
    return out


def elastic_setup(shape, bc, h, dt, rho, vp, vs, store_fmt, comp, P0=1.0, arith_fmt=None,
                  stencil_fmt=None, init=None, coef_fmt=None, pair_stencil=False):
    """Ready-to-run ElasticState from physical inputs. init: dict field -> array
    (velocities in m/s, stresses in Pa). coef_fmt: round the multipliers to
    this format instead of the storage format; pair_stencil: see elastic_cfg."""
    cfg = elastic_cfg(shape, bc, store_fmt, comp, arith_fmt, stencil_fmt, pair_stencil)
    st = ElasticState(cfg)
    ccfg = cfg if coef_fmt is None else elastic_cfg(shape, bc, coef_fmt, comp)
    coef, Z0, ok = elastic_coefficients(ccfg, h, dt, rho, vp, vs)
    if not ok:
        raise ValueError("elastic multiplier outside the storage format's range")
    st.coef, st.Z0, st.P0, st.h, st.dt = coef, Z0, P0, h, dt
    for name, arr in (init or {}).items():
        if name in ("vx", "vy"):
            st.f[name] = scale_velocity(arr, Z0, P0, store_fmt).reshape(st.shape)
        else:
            st.f[name] = scale_pressure(arr, P0, store_fmt).reshape(st.shape)
    st.apply_walls()
    return st
