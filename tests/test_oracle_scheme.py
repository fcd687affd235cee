"""Pins for the oracle's time stepping (Section 3, Algorithms 1 and 2).

* Exact discrete energy conservation of the FP64 scheme (Section 3 states the
  discrete system conserves energy; the energy used is the leapfrog form
  E^{n+1/2} = sum v^2/a + sum p^n p^{n+1}/b with the scheme's own coefficients).
* Second-order convergence in time to an analytic standing mode.
* Exact mirror / transpose symmetry in every precision for a centred Gaussian.
* Special cases: zero stays zero; constant pressure with periodic walls stays.
"""
import numpy as np
import pytest

import oracle as O
from paper_2310_00236_gb300 import inputs


def _drift(E):
    return float(np.max(np.abs(E - E[0])) / abs(E[0]))


def test_energy_conserved_fp64_2d_gaussian_2000_steps(oracle_lib):
    """256^2 cells, rho = c = 1, p = 0 walls, CFL 0.5, 2000 steps."""
    w = inputs.acoustic_2d_gaussian(256, 2000)
    st = O.acoustic_setup(w["shape"], (O.BC_RIGID,) * 2, w["h"], w["dt"], w["rho"], w["c"],
                          O.FP64, 0, p0=w["p0"])
    _, E = st.run(w["steps"], energy=True)
    assert _drift(E) <= 1e-12
    assert E[0] > 0


def test_energy_conserved_fp64_variable_media(oracle_lib):
    """Variable density and speed, mixed boundaries, 2D and 3D."""
    rng = np.random.default_rng(7)
    for shape, bc in (((48, 40), (O.BC_RIGID, O.BC_PERIODIC)),
                      ((20, 18, 16), (O.BC_PERIODIC, O.BC_RIGID, O.BC_RIGID))):
        nd = len(shape)
        h = 5.0
        c = inputs.smooth_random_field(shape, 3, 3.0, 1500.0, 4500.0)
        rho = inputs.smooth_random_field(shape, 4, 3.0, 1000.0, 2500.0)
        dt = 0.45 * h / 4500.0 / np.sqrt(nd / 2.0)
        p0 = inputs.gaussian(shape, h, 3 * h) + 0.1 * rng.standard_normal(c.shape)
        v0 = [0.01 * rng.standard_normal(c.shape) for _ in range(nd)]
        st = O.acoustic_setup(shape, bc, h, dt, rho, c, O.FP64, 0, P0=1.0, p0=p0, v0=v0)
        _, E = st.run(300, energy=True)
        assert _drift(E) <= 1e-12, (shape, _drift(E))


def test_energy_formula_recomputed_outside_the_oracle(oracle_lib):
    """The oracle's energy equals sum v^2/a + sum p^n p^{n+1}/b recomputed here
    with numpy from the stepped states, and weighting with coefficients that are
    not the ones the scheme rounded (here fp16-rounded vs exact) shows drift, so
    the conservation pin depends on the weights being the scheme's own."""
    n = 64
    h = 1.0 / n
    dt = 0.37 * h
    c = inputs.smooth_random_field((n, n), 5, 4.0, 0.6, 1.0)
    st = O.acoustic_setup((n, n), (O.BC_RIGID,) * 2, h, dt, np.ones((n, n)), c, O.FP64, 0,
                          p0=inputs.gaussian((n, n), h, 0.1))
    b_exact = dt * c * c / (1.0 * h)      # Z0 = 1 here
    st16 = [O.round_to(x, O.FP16) for x in (st.a[0], st.a[1], st.b)]
    st.a[0], st.a[1], st.b = st16
    E_orc, E_ext, E_wrong = [], [], []
    for _ in range(300):
        p_old = st.p.copy()
        _, E = st.run(1, energy=True)
        E_orc.append(E[0])
        kin = np.sum(st.v[0] ** 2 / st.a[0]) + np.sum(st.v[1] ** 2 / st.a[1])
        E_ext.append(kin + np.sum(p_old * st.p / st.b))
        E_wrong.append(kin + np.sum(p_old * st.p / b_exact))
    E_orc, E_ext, E_wrong = map(np.array, (E_orc, E_ext, E_wrong))
    np.testing.assert_allclose(E_orc, E_ext, rtol=1e-13)
    assert _drift(E_orc) <= 1e-12
    assert _drift(E_wrong) > 1e-7


def _standing_mode(N, cfl, T, k=1, l=2):
    """p = cos(w t) sin(k pi x) sin(l pi y) on [0,1]^2, p = 0 walls, rho = c = 1.
    With rho dv/dt = grad p (Eq. 1 sign convention), v = sin(w t)/w grad(sin sin)."""
    h = 1.0 / N
    dt = cfl * h
    nsteps = int(round(T / dt))
    w = np.pi * np.hypot(k, l)
    x = np.arange(N) * h
    xh = x + 0.5 * h
    X, Y = np.meshgrid(x, x, indexing="xy")
    p0 = np.sin(k * np.pi * X) * np.sin(l * np.pi * Y)
    t_half = -0.5 * dt
    Xh, Yn = np.meshgrid(xh, x, indexing="xy")
    vx = np.sin(w * t_half) / w * k * np.pi * np.cos(k * np.pi * Xh) * np.sin(l * np.pi * Yn)
    Xn, Yh = np.meshgrid(x, xh, indexing="xy")
    vy = np.sin(w * t_half) / w * l * np.pi * np.sin(k * np.pi * Xn) * np.cos(l * np.pi * Yh)
    st = O.acoustic_setup((N, N), (O.BC_RIGID,) * 2, h, dt, np.ones((N, N)), np.ones((N, N)),
                          O.FP64, 0, p0=p0, v0=[vx, vy])
    st.run(nsteps)
    exact = np.cos(w * nsteps * dt) * p0
    return np.max(np.abs(st.p - exact))


def test_second_order_convergence_standing_mode(oracle_lib):
    Ns = [32, 64, 128]
    errs = [_standing_mode(N, 0.5, 0.5) for N in Ns]
    slopes = np.diff(np.log(errs)) / np.diff(np.log([1.0 / N for N in Ns]))
    assert np.all(np.abs(slopes - 2.0) < 0.1), (errs, slopes)


def test_fourth_order_in_space_at_small_cfl(oracle_lib):
    """At a tiny time step the spatial 4th-order error dominates."""
    Ns = [16, 32]
    errs = [_standing_mode(N, 0.02, 0.25, k=2, l=3) for N in Ns]
    slope = np.log(errs[0] / errs[1]) / np.log(2.0)
    assert 3.6 < slope < 4.4, (errs, slope)


VARIANTS = [(O.FP16, 0, None), (O.FP16, 3, None), (O.FP16, 6, None), (O.BF16, 3, None),
            (O.FP32, 0, None), (O.FP16, 3, O.FP32), (O.FP16, 0, O.FP32), (O.BF16, 3, O.FP32)]


@pytest.mark.parametrize("fmt,comp,arith", VARIANTS)
def test_centred_gaussian_symmetries_exact(oracle_lib, fmt, comp, arith):
    N = 32
    w = inputs.acoustic_2d_gaussian(N, 60, cfl=0.45, sigma=0.1)
    st = O.acoustic_setup(w["shape"], (O.BC_RIGID,) * 2, w["h"], w["dt"], w["rho"], w["c"],
                          fmt, comp, arith_fmt=arith, p0=w["p0"])
    st.run(60)
    p, vx, vy = st.p, st.v[0], st.v[1]
    assert np.any(p != 0)
    # transpose symmetry
    assert np.array_equal(p, p.T)
    assert np.array_equal(vx, vy.T)
    assert np.array_equal(st.tp, st.tp.T)
    # mirror about the centre node N/2: p[i] = p[N - i], vx[i] = -vx[N - 1 - i]
    idx = np.arange(1, N)
    assert np.array_equal(p[:, idx], p[:, N - idx])
    assert np.array_equal(vx[:, :], -vx[:, ::-1])
    assert np.array_equal(st.tv[0][:, :], -st.tv[0][:, ::-1])


@pytest.mark.parametrize("fmt,comp,arith", VARIANTS)
def test_zero_state_stays_zero(oracle_lib, fmt, comp, arith):
    shape = (12, 10)
    st = O.acoustic_setup(shape, (O.BC_RIGID, O.BC_PERIODIC), 0.1, 0.02,
                          np.ones((10, 12)), np.ones((10, 12)), fmt, comp, arith_fmt=arith)
    st.run(20)
    for f in [st.p, st.tp, *st.v, *st.tv]:
        assert not np.any(f)


@pytest.mark.parametrize("fmt,comp,arith", VARIANTS)
def test_constant_pressure_periodic_stays(oracle_lib, fmt, comp, arith):
    shape = (12, 10, 8)
    ones = np.ones((8, 10, 12))
    st = O.acoustic_setup(shape, (O.BC_PERIODIC,) * 3, 0.1, 0.02, ones, ones, fmt, comp,
                          arith_fmt=arith, p0=0.71 * ones)
    p_init = st.p.copy()
    st.run(15)
    assert np.array_equal(st.p, p_init)
    for f in [st.tp, *st.v, *st.tv]:
        assert not np.any(f)


def test_fp64_equals_fp32_to_roundoff(oracle_lib):
    """FP32 tracks FP64 closely on a short run (Section 3: fp32 is adequate)."""
    w = inputs.acoustic_2d_gaussian(64, 200)
    r = {}
    for fmt in (O.FP64, O.FP32):
        st = O.acoustic_setup(w["shape"], (O.BC_RIGID,) * 2, w["h"], w["dt"], w["rho"], w["c"],
                              fmt, 0, p0=w["p0"])
        st.run(200)
        r[fmt] = st.p
    err = np.linalg.norm(r[O.FP32] - r[O.FP64]) / np.linalg.norm(r[O.FP64])
    assert 0 < err < 1e-5


def test_results_independent_of_thread_count(oracle_lib):
    """The OpenMP loops write disjoint points and combine the energy partial
    sums in a fixed order, so one thread and all threads give identical bits
    (the CPU baseline times both)."""
    w = inputs.acoustic_3d_random(n=24, sigma_cells=2.0, ic_sigma_cells=2.0, smooth_dtype=np.float64)
    out = []
    before = O.set_threads()
    try:
        for t in (1, max(2, before)):
            O.set_threads(t)
            st = O.acoustic_setup(w["shape"], (1, 0, 1), w["h"], w["dt"], w["rho"], w["c"], O.FP16, 3,
                                  p0=w["p0"])
            _, E = st.run(6, energy=True)
            out.append((st.p.copy(), st.v[0].copy(), np.array(E)))
    finally:
        O.set_threads(before)
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def _standing_mode_physical(N, cfl, nsteps, rho, c, P0, Pamp, L, k=1, l=2):
    """The standing mode of `_standing_mode` in physical units on [0, L]^2:
    p = Pamp cos(w t) sin(k pi x / L) sin(l pi y / L), rho dv/dt = grad p,
    so v = Pamp sin(w t) / (rho w) grad(sin sin), w = c pi sqrt(k^2 + l^2) / L.
    Returns the largest errors of p (relative to Pamp) and of v (relative to
    Pamp / (rho c)) after nsteps, the oracle's state read back as
    p = P0 p^ and v = P0 v^ / Z0."""
    h = L / N
    dt = cfl * h / c
    w = c * np.pi * np.hypot(k, l) / L
    x = np.arange(N) * h
    xh = x + 0.5 * h

    def fields(t_p, t_v):
        X, Y = np.meshgrid(x, x, indexing="xy")
        p = Pamp * np.cos(w * t_p) * np.sin(k * np.pi * X / L) * np.sin(l * np.pi * Y / L)
        Xh, Yn = np.meshgrid(xh, x, indexing="xy")
        vx = (Pamp * np.sin(w * t_v) / (rho * w) * (k * np.pi / L) * np.cos(k * np.pi * Xh / L)
              * np.sin(l * np.pi * Yn / L))
        Xn, Yh = np.meshgrid(x, xh, indexing="xy")
        vy = (Pamp * np.sin(w * t_v) / (rho * w) * (l * np.pi / L) * np.sin(k * np.pi * Xn / L)
              * np.cos(l * np.pi * Yh / L))
        return p, vx, vy

    p0, vx0, vy0 = fields(0.0, -0.5 * dt)
    st = O.acoustic_setup((N, N), (O.BC_RIGID,) * 2, h, dt, np.full((N, N), rho), np.full((N, N), c),
                          O.FP64, 0, P0=P0, p0=p0, v0=[vx0, vy0])
    st.run(nsteps)
    pe, vxe, vye = fields(nsteps * dt, (nsteps - 0.5) * dt)
    ep = np.max(np.abs(st.p * P0 - pe)) / Pamp
    vscale = Pamp / (rho * c)
    ev = max(np.max(np.abs(st.v[0] * P0 / st.Z0 - vxe)), np.max(np.abs(st.v[1] * P0 / st.Z0 - vye))) / vscale
    return ep, ev


def test_scaled_variables_reproduce_physical_units(oracle_lib):
    """Scaled variables (Section 3: p^ = p / P0, v^ = v Z0 / P0, Z0 = max rho
    * max c) with rho = 1800 kg/m^3, c = 2500 m/s, P0 = 3e4 Pa on a 640 m box
    give, read back in physical units, the same relative error against the
    analytic standing mode as the nondimensional problem (rho = c = L = 1,
    P0 = 1), which is the same discrete problem up to rounding; the error is
    the scheme's own (second order, about 1e-3 here). A wrong Z0 or P0 in the
    scaling of p, v or of the multipliers changes the physical solution by
    orders of magnitude."""
    N, cfl, nsteps = 64, 0.5, 64
    ep, ev = _standing_mode_physical(N, cfl, nsteps, 1800.0, 2500.0, 3.0e4, 2.0e5, 640.0)
    ep1, ev1 = _standing_mode_physical(N, cfl, nsteps, 1.0, 1.0, 1.0, 1.0, 1.0)
    assert 1e-5 < ep1 < 1e-2 and 1e-5 < ev1 < 1e-2, (ep1, ev1)
    assert abs(ep - ep1) <= 1e-9 + 1e-6 * ep1, (ep, ep1)
    assert abs(ev - ev1) <= 1e-9 + 1e-6 * ev1, (ev, ev1)


@pytest.mark.parametrize("shape", [(12, 10), (10, 9, 8)])
def test_point_source_first_step_closed_form(oracle_lib, shape):
    """A point source of volume-injection rate w (p_t = rho c^2 (div v + w
    delta), the delta discretised as 1/h^d, Algorithm 1's source line) in a
    zero state: after one step v is still zero and p at the source node has
    grown by dt rho c^2 w / h^d, in physical units (P0 p^), whatever P0 and
    the medium; nothing else moved. This fixes the source scaling
    s^ = w Z0 / (P0 h^(d-1)) together with the multiplier b."""
    nd = len(shape)
    h, rho0, c0, P0, w = 7.0, 1800.0, 2400.0, 3.0e4, 0.37
    rho = np.full(tuple(shape[::-1]), rho0)
    c = np.full(tuple(shape[::-1]), c0)
    rho.flat[5] = 2200.0                      # Z0 = max rho * max c differs from rho0 c0
    dt = 0.3 * h / c0
    st = O.acoustic_setup(shape, (O.BC_RIGID,) * nd, h, dt, rho, c, O.FP64, 0, P0=P0)
    src = tuple(s // 2 for s in shape)
    q = int(np.ravel_multi_index(src[::-1], tuple(shape[::-1])))
    st.src_index = q
    st.src = O.scale_source(np.array([w, 0.0]), st.Z0, P0, h, nd, O.FP64)
    st.run(1)
    expect = dt * rho0 * c0 * c0 * w / h ** nd
    np.testing.assert_allclose(st.p.flat[q] * P0, expect, rtol=1e-14)
    assert np.count_nonzero(st.p) == 1
    assert all(np.count_nonzero(v) == 0 for v in st.v[:nd])


def _standing_mode_energy(N, L=640.0, rho=1800.0, c=2500.0, P0=3.0e4, Pamp=2.0e5, k=1, l=2):
    """Relative gap between the oracle's energy of the physical-units standing
    mode (scaled energy times energy_factor) and the continuous energy
    1/2 int (p^2 / (rho c^2) + rho |v|^2) = Pamp^2 L^2 / (8 rho c^2) per unit
    depth (at t = 0 all of it is in p)."""
    h = L / N
    dt = 0.5 * h / c
    w = c * np.pi * np.hypot(k, l) / L
    x = np.arange(N) * h
    xh = x + 0.5 * h
    X, Y = np.meshgrid(x, x, indexing="xy")
    p0 = Pamp * np.sin(k * np.pi * X / L) * np.sin(l * np.pi * Y / L)
    tv = -0.5 * dt
    Xh, Yn = np.meshgrid(xh, x, indexing="xy")
    Xn, Yh = np.meshgrid(x, xh, indexing="xy")
    vx = Pamp * np.sin(w * tv) / (rho * w) * (k * np.pi / L) * np.cos(k * np.pi * Xh / L) * np.sin(l * np.pi * Yn / L)
    vy = Pamp * np.sin(w * tv) / (rho * w) * (l * np.pi / L) * np.sin(k * np.pi * Xn / L) * np.cos(l * np.pi * Yh / L)
    st = O.acoustic_setup((N, N), (O.BC_RIGID,) * 2, h, dt, np.full((N, N), rho), np.full((N, N), c),
                          O.FP64, 0, P0=P0, p0=p0, v0=[vx, vy])
    _, E = st.run(20, energy=True)
    E = np.asarray(E) * O.energy_factor(h, dt, P0, st.Z0, 2)
    return E[0] / (Pamp ** 2 * L ** 2 / (8.0 * rho * c * c)) - 1.0, _drift(E)


def test_energy_in_physical_units_converges_to_continuous(oracle_lib):
    """The discrete energy converted with energy_factor (0.5 h^(d-1) P0^2 dt /
    Z0) approaches the continuous energy of the standing mode at second order
    (rho, c, P0 far from 1, so a wrong power of h, P0 or Z0 in the factor is
    off by orders of magnitude), and is conserved."""
    e64, d64 = _standing_mode_energy(64)
    e128, d128 = _standing_mode_energy(128)
    assert abs(e64) < 2e-3 and abs(e128) < abs(e64) / 3.0, (e64, e128)
    assert d64 <= 1e-12 and d128 <= 1e-12
