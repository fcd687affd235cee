"""Pins for the oracle's elastic velocity-stress scheme (Eq. 2, Appendix A).

* Brute-force operators on tiny grids against dense matrices assembled here
  from the printed stencil weights and the boundary images, and the exact
  negative-transpose (skew) structure on the free unknowns.
* Exact FP64 energy conservation with periodic, rigid and free faces.
* Reduction to the (separately pinned) acoustic oracle: a plane P wave along x
  is the 1D acoustic problem with a = bx, b = l2m; a plane S wave is the one
  with a = by, b = mu.
* Mirror symmetry, zero state, and the paper's compensation finding in the
  elastic case (Appendix A: fp16 without compensation loses energy, with
  sum_6op it does not).
* The analytic standing P wave in physical units (rho, vp, P0 far from 1):
  the Z0 / P0 scaling of stresses, velocities and multipliers.
* The free surface (Appendix A: free surface in y) is traction free: a
  vertically incident P pulse comes back with syy reversed and v_y doubled on
  the surface (a rigid wall keeps the sign), and the analytic Rayleigh wave of
  a homogeneous half-space is reproduced with second-order convergence.
"""
from scipy.optimize import brentq
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2310_00236_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PER, RIG, FREE = O.EBC_PERIODIC, O.EBC_RIGID, O.EBC_FREE


def _weights():
    w = {}
    with open(os.path.join(GOLDEN, "stencil_weights.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            off, wt = line.split()
            w[float(off)] = float(Fraction(wt))
    return w


def _ext(N, lo, hi, node, odd, odd_free):
    """Dense image map from N stored values to positions -3..N+2. Rigid walls
    sit on the half points -1/2 and N-1/2 (parity `odd`); a free surface sits
    on the node 0 (parity `odd_free`: odd for the stresses that carry a y
    traction, even for the velocities)."""
    E = np.zeros((N + 6, N))
    for r in range(N + 6):
        m = r - 3
        if 0 <= m < N:
            E[r, m] = 1.0
            continue
        bc = lo if m < 0 else hi
        if bc == PER:
            E[r, m % N] = 1.0
        elif bc == FREE:
            # mirror about y = 0: node -m <-> m, half point -(m + 1/2) <-> m + 1/2
            E[r, -m if node else -1 - m] = -1.0 if odd_free else 1.0
        elif node:
            E[r, (-1 - m) if m < 0 else (2 * N - 1 - m)] = -1.0 if odd else 1.0
        else:
            if m == -1:
                if not odd:
                    E[r, 0] = 1.0
                continue
            E[r, (-2 - m) if m < 0 else (2 * N - 2 - m)] = -1.0 if odd else 1.0
    return E


def _diff(N, lo, hi, src_node, odd, odd_free):
    """Undivided derivative of a field that is node-type (src_node) or
    half-type along the axis, evaluated at the other kind of point."""
    w = _weights()
    E = _ext(N, lo, hi, src_node, odd, odd_free)
    D = np.zeros((N, N))
    for m in range(N):
        first = m - 1 if src_node else m - 2
        taps = dict(zip(range(first, first + 4), (w[-1.5], w[-0.5], w[0.5], w[1.5])))
        for pos, wt in taps.items():
            D[m] += wt * E[pos + 3]
    return D


def _along(mat, ax, shape):
    nx, ny = shape
    return np.kron(np.eye(ny), mat) if ax == 0 else np.kron(mat, np.eye(nx))


FIELDS = ("vx", "vy", "sxx", "syy", "sxy")
# (target, source field, axis, source node-type along axis, odd about rigid
# walls); the parity about a free surface is odd for stresses, even for velocities
MAPS = [("vx", "sxx", 0, True, False), ("vx", "sxy", 1, False, True),
        ("vy", "sxy", 0, False, True), ("vy", "syy", 1, True, False),
        ("sxx", "vx", 0, False, True), ("syy", "vy", 1, False, True),
        ("sxy", "vy", 0, True, False), ("sxy", "vx", 1, True, False)]


def _impulse_maps(shape, bc):
    """Impulse responses of one FP64 step with unit multipliers, separated
    by switching off the other half step (its multipliers set to zero)."""
    nx, ny = shape
    npts = nx * ny
    cfg = O.elastic_cfg(shape, bc, O.FP64, 0)
    out = {}
    for tgt, src, ax, node, odd in MAPS:
        M = np.zeros((npts, npts))
        for q in range(npts):
            st = O.ElasticState(cfg)
            for k in st.coef:
                st.coef[k] = np.zeros(st.shape)
            st.f[src].flat[q] = 1.0
            if tgt in ("vx", "vy"):
                st.coef["bx" if tgt == "vx" else "by"][:] = 1.0
            elif tgt == "sxy":
                st.coef["mu"][:] = 1.0
            else:
                st.coef["l2m"][:] = 1.0
            st.run(1)
            M[:, q] = st.f[tgt].ravel() - (st.f[src].ravel() if src == tgt else 0)
        out[(tgt, src)] = M
    return out


CASES = [((8, 8), (RIG, RIG, FREE, RIG)), ((8, 7), (PER, PER, FREE, RIG)),
         ((7, 8), (RIG, RIG, RIG, RIG)), ((8, 8), (PER, PER, PER, PER))]


def _held(shape, bc, name):
    """Mask of points a boundary holds at zero: the normal velocity and the
    shear stress on the stored points of a rigid wall, syy on a free surface."""
    nx, ny = shape
    m = np.zeros((ny, nx), bool)
    if bc[1] == RIG and name in ("vx", "sxy"):
        m[:, nx - 1] = True
    if bc[3] == RIG and name in ("vy", "sxy"):
        m[ny - 1, :] = True
    if bc[2] == FREE and name == "syy":
        m[0, :] = True
    return m.ravel()


def _weight(shape, bc, name):
    """Energy weight of each point: 1/2 for vx and sxx on the row of a free
    surface (the mirror plane of the images), 1 elsewhere."""
    nx, ny = shape
    w = np.ones((ny, nx))
    if bc[2] == FREE and name in ("vx", "sxx"):
        w[0, :] = 0.5
    return w.ravel()


@pytest.mark.parametrize("shape,bc", CASES)
def test_elastic_operators_brute_force_and_skew(oracle_lib, shape, bc):
    maps = _impulse_maps(shape, bc)
    for tgt, src, ax, node, odd in MAPS:
        N = shape[ax]
        odd_free = src.startswith("s")
        ref = _along(_diff(N, bc[2 * ax], bc[2 * ax + 1], node, odd, odd_free), ax, shape)
        np.testing.assert_array_equal(maps[(tgt, src)], ref, err_msg=f"{src}->{tgt}")
    # skew: the stress-to-velocity map G is minus the adjoint of the
    # velocity-to-strain-rate map D in the weighted inner products, on the
    # unknowns not held at zero: W_v G = -(W_s D)^T
    pairs = [(("vx", "sxx"), ("sxx", "vx")), (("vx", "sxy"), ("sxy", "vx")),
             (("vy", "sxy"), ("sxy", "vy")), (("vy", "syy"), ("syy", "vy"))]
    for (a, b), (c, d) in pairs:
        fa, fb = ~_held(shape, bc, a), ~_held(shape, bc, b)
        G = maps[(a, b)][np.ix_(fa, fb)]
        D = maps[(c, d)][np.ix_(fb, fa)]
        wa, wb = _weight(shape, bc, a)[fa], _weight(shape, bc, b)[fb]
        np.testing.assert_array_equal(wa[:, None] * G, -(wb[:, None] * D).T, err_msg=f"{a}<-{b}")


def _layered(shape, h):
    nx, ny = shape
    y = np.arange(ny)
    vp = np.where(y < ny // 3, 2000.0, np.where(y < 2 * ny // 3, 3000.0, 4000.0))
    rho = np.where(y < ny // 3, 2000.0, np.where(y < 2 * ny // 3, 2300.0, 2600.0))
    vp = np.repeat(vp[:, None], nx, 1)
    rho = np.repeat(rho[:, None], nx, 1)
    return rho, vp, vp / 1.73


@pytest.mark.parametrize("bc", [(RIG, RIG, FREE, RIG), (PER, PER, FREE, RIG),
                                (PER, PER, PER, PER), (RIG, RIG, RIG, RIG)])
def test_elastic_energy_conserved_fp64(oracle_lib, bc):
    shape = (40, 36)
    h = 3.0
    rho, vp, vs = _layered(shape, h)
    dt = 0.5 * h / 4000.0
    rng = np.random.default_rng(3)
    init = {"sxx": rng.standard_normal(rho.shape), "sxy": rng.standard_normal(rho.shape),
            "vy": rng.standard_normal(rho.shape) / 1e7}
    st = O.elastic_setup(shape, bc, h, dt, rho, vp, vs, O.FP64, 0, init=init)
    _, E = st.run(800, energy=True)
    assert np.max(np.abs(E - E[0])) / E[0] <= 1e-12


def test_elastic_reduces_to_acoustic_for_plane_waves(oracle_lib):
    """A wave independent of y in a periodic homogeneous medium: (vx, sxx) is
    the 1D acoustic problem with a = bx and b = l2m; (vy, sxy) with a = by and
    b = mu. Same values in fp16 with sum_3op, step for step."""
    nx, ny = 48, 8
    h = 2.0
    rho = np.full((ny, nx), 2200.0)
    vp = np.full((ny, nx), 3000.0)
    vs = vp / 1.73
    dt = 0.45 * h / 3000.0
    x = np.arange(nx) * h
    prof = np.exp(-((x - 40.0) / 8.0) ** 2)
    init = {"sxx": np.repeat(prof[None, :], ny, 0), "sxy": np.repeat(prof[None, :], ny, 0)}
    st = O.elastic_setup((nx, ny), (PER,) * 4, h, dt, rho, vp, vs, O.FP16, 3, init=init)
    # acoustic 2D with the elastic multipliers, uniform in y
    cfg = O.acoustic_cfg((nx, ny), (O.BC_PERIODIC, O.BC_PERIODIC), O.FP16, 3)
    acP = O.AcousticState(cfg)
    acP.p = st.f["sxx"].copy()
    acP.a = [st.coef["bx"].copy(), st.coef["bx"].copy(), np.zeros((ny, nx))]
    acP.b = st.coef["l2m"].copy()
    st.run(60)
    acP.run(60)
    np.testing.assert_array_equal(st.f["vx"], acP.v[0])
    np.testing.assert_array_equal(st.f["sxx"], acP.p)
    np.testing.assert_array_equal(st.t["sxx"], acP.tp)
    # the S wave (vy, sxy) has the node and half-point roles swapped in x: it
    # is the acoustic problem with p <- vy (nodes), v <- sxy (half points),
    # a <- mu and b <- by, since vy' = by Dx(sxy) and sxy' = mu Dx(vy)
    acS = O.AcousticState(cfg)
    st2 = O.elastic_setup((nx, ny), (PER,) * 4, h, dt, rho, vp, vs, O.FP16, 3,
                          init={"vy": np.repeat(prof[None, :], ny, 0) / 3e6})
    acS.p = st2.f["vy"].copy()
    acS.a = [st2.coef["mu"].copy(), st2.coef["mu"].copy(), np.zeros((ny, nx))]
    acS.b = st2.coef["by"].copy()
    # sxy starts at zero, so the elastic v_y half step of step 1 changes
    # nothing and sxy after k elastic steps equals the acoustic "velocity"
    # after k steps (both come from the same k-1 updates of vy)
    st2.run(60)
    acS.run(60)
    np.testing.assert_array_equal(st2.f["sxy"], acS.v[0])
    assert np.any(st2.f["vy"] != 0)


def test_elastic_mirror_symmetry_exact(oracle_lib):
    """Symmetric initial stresses about the vertical line x = (N-1)/2 in a
    domain with rigid side walls: vy and the normal stresses stay mirror
    symmetric and vx antisymmetric, bit for bit, in fp16 + sum_6op."""
    nx, ny = 31, 24
    h = 3.0
    rho, vp, vs = _layered((nx, ny), h)
    dt = 0.5 * h / 4000.0
    x = np.arange(nx) - (nx - 1) / 2
    y = np.arange(ny) - 8.0
    X, Y = np.meshgrid(x, y)
    g = np.exp(-(X ** 2 + Y ** 2) / 10.0) * 1e5
    st = O.elastic_setup((nx, ny), (RIG, RIG, FREE, RIG), h, dt, rho, vp, vs, O.FP16, 6,
                         P0=1e5, init={"sxx": g, "syy": g})
    st.run(80)
    for name in ("vy", "sxx", "syy"):
        np.testing.assert_array_equal(st.f[name], st.f[name][:, ::-1])
    # vx at i+1/2 mirrors to index nx-2-i; column nx-1 is held at zero
    np.testing.assert_array_equal(st.f["vx"][:, : nx - 1], -st.f["vx"][:, nx - 2::-1])
    assert np.any(st.f["vx"] != 0)


def test_elastic_fp16_compensation_finding(oracle_lib):
    """Appendix A: without compensation fp16 loses energy; sum_6op keeps it
    (small CFL, pulse in a layered medium with a free top)."""
    shape = (48, 40)
    h = 3.0
    rho, vp, vs = _layered(shape, h)
    dt = 0.02 * h / 4000.0
    x = np.arange(shape[0]) * h
    y = np.arange(shape[1]) * h
    X, Y = np.meshgrid(x, y)
    g = np.exp(-((X - 72.0) ** 2 + (Y - 60.0) ** 2) / (2 * 9.0 ** 2)) * 1e6
    res = {}
    for comp in (0, 3, 6):
        st = O.elastic_setup(shape, (PER, PER, FREE, RIG), h, dt, rho, vp, vs, O.FP16, comp,
                             P0=1e6, init={"sxx": g, "syy": g})
        _, E = st.run(3000, energy=True)
        res[comp] = (E - E[0]) / E[0]
    q = res[0][[750, 1500, 2250, 2999]]
    assert np.all(np.diff(q) < 0) and res[0][-1] < -0.01       # monotone loss
    assert np.max(np.abs(res[6])) < 0.05 * -res[0][-1]
    # "sum_3op gives very similar results" (Appendix A)
    assert np.max(np.abs(res[3] - res[6])) < 0.05 * -res[0][-1]


def test_elastic_zero_state_stays_zero(oracle_lib):
    shape = (12, 10)
    rho, vp, vs = _layered(shape, 3.0)
    for fmt, comp in ((O.FP16, 3), (O.BF16, 6), (O.FP32, 0)):
        st = O.elastic_setup(shape, (RIG, RIG, FREE, RIG), 3.0, 3.0e-4, rho, vp, vs, fmt, comp)
        st.run(10)
        for k in O.ELASTIC_FIELDS:
            assert not np.any(st.f[k]) and not np.any(st.t[k])


def _standing_p_wave(nx, cfl, nsteps, rho, vp, P0, S, L):
    """Standing P wave along x in a periodic homogeneous medium, independent
    of y, in physical units: with rho dvx/dt = d(sxx)/dx, d(sxx)/dt =
    (lambda + 2 mu) d(vx)/dx and d(syy)/dt = lambda d(vx)/dx,
      sxx = S cos(w t) cos(k x),  syy = lambda / (lambda + 2 mu) sxx,
      vx = -S k / (rho w) sin(w t) sin(k x),  w = vp k,  k = 2 pi / L,
    with the stresses at nodes i h and vx at (i + 1/2) h. Returns the largest
    errors after nsteps of sxx and syy (relative to S) and of vx (relative to
    S / (rho vp)), the state read back as P0 s^ and P0 v^ / Z0."""
    ny = 8
    h = L / nx
    vs = vp / 1.73
    mu = rho * vs * vs
    lam = rho * vp * vp - 2.0 * mu
    dt = cfl * h / vp
    k = 2.0 * np.pi / L
    w = vp * k
    x = np.arange(nx) * h
    xh = x + 0.5 * h

    def fields(ts, tv):
        sxx = S * np.cos(w * ts) * np.cos(k * x)
        vx = -S * k / (rho * w) * np.sin(w * tv) * np.sin(k * xh)
        return [np.repeat(f[None, :], ny, 0) for f in (sxx, lam / (lam + 2 * mu) * sxx, vx)]

    sxx0, syy0, vx0 = fields(0.0, -0.5 * dt)
    full = np.full((ny, nx), 1.0)
    st = O.elastic_setup((nx, ny), (PER,) * 4, h, dt, rho * full, vp * full, vs * full, O.FP64, 0,
                         P0=P0, init={"sxx": sxx0, "syy": syy0, "vx": vx0})
    st.run(nsteps)
    sxx, syy, vx = fields(nsteps * dt, (nsteps - 0.5) * dt)
    es = max(np.max(np.abs(st.f["sxx"] * P0 - sxx)), np.max(np.abs(st.f["syy"] * P0 - syy))) / S
    ev = np.max(np.abs(st.f["vx"] * P0 / st.Z0 - vx)) / (S / (rho * vp))
    return es, ev


def test_elastic_scaled_variables_reproduce_physical_units(oracle_lib):
    """Scaled elastic variables (s^ = s / P0, v^ = v Z0 / P0, Z0 = max rho *
    max vp) with rho = 2200 kg/m^3, vp = 3000 m/s, P0 = 1e5 Pa on a 256 m
    periodic box give, read back in physical units, the same relative errors
    against the analytic standing P wave as the nondimensional problem (rho =
    vp = L = 1, P0 = 1), which is the same discrete problem up to rounding;
    the errors are the scheme's own (about 1e-4 here). A wrong Z0 or P0 in
    the scaling of stresses, velocities or multipliers fails it."""
    nx, cfl, nsteps = 64, 0.5, 96
    es, ev = _standing_p_wave(nx, cfl, nsteps, 2200.0, 3000.0, 1.0e5, 3.0e6, 256.0)
    es1, ev1 = _standing_p_wave(nx, cfl, nsteps, 1.0, 1.0, 1.0, 1.0, 1.0)
    assert 1e-7 < es1 < 1e-2 and 1e-7 < ev1 < 1e-2, (es1, ev1)
    assert abs(es - es1) <= 1e-9 + 1e-6 * es1, (es, es1)
    assert abs(ev - ev1) <= 1e-9 + 1e-6 * ev1, (ev, ev1)


def test_elastic_vy_source_first_step_closed_form(oracle_lib):
    """The vertical force source enters v_y's increment outside the 1/rho
    factor (Eq. 2): from a zero state, one step leaves v_y = w dt / h^2 at the
    source point in physical units (P0 v^ / Z0) and v_x zero everywhere (the
    stresses of that step move only through the derivatives of that v_y).
    This fixes s^ = w dt Z0 / (P0 h^2)."""
    shape = (12, 10)
    h, P0, w = 3.0, 1.0e5, 2.5e3
    rho, vp, vs = _layered(shape, h)
    dt = 0.5 * h / 4000.0
    st = O.elastic_setup(shape, (RIG, RIG, FREE, RIG), h, dt, rho, vp, vs, O.FP64, 0, P0=P0)
    i, j = 6, 5
    st.src_index = i + shape[0] * j
    st.src = O.elastic_scale_source(np.array([w, 0.0]), dt, st.Z0, P0, h, O.FP64)
    st.run(1)
    vy = st.f["vy"] * P0 / st.Z0
    np.testing.assert_allclose(vy[j, i], w * dt / h ** 2, rtol=1e-14)
    assert np.count_nonzero(st.f["vy"]) == 1 and np.count_nonzero(st.f["vx"]) == 0


def _p_wave_energy_gap(nx, L=256.0, rho=2200.0, vp=3000.0, P0=1.0e5, S=3.0e6):
    """Relative gap between the elastic energy of the standing P wave, scaled
    energy times 0.5 h P0^2 dt / Z0, and the continuous energy: uniaxial strain
    (syy = lambda / (lambda + 2 mu) sxx, e_yy = 0) stores sxx^2 / (2 (lambda +
    2 mu)) per unit area, S^2 L H / (4 (lambda + 2 mu)) in the box L x H at t = 0."""
    ny = 8
    h = L / nx
    vs = vp / 1.73
    mu = rho * vs * vs
    lam = rho * vp * vp - 2.0 * mu
    dt = 0.5 * h / vp
    k = 2.0 * np.pi / L
    w = vp * k
    x = np.arange(nx) * h
    sxx = S * np.cos(k * x)
    vx = -S * k / (rho * w) * np.sin(w * (-0.5 * dt)) * np.sin(k * (x + 0.5 * h))

    def rep(f):
        return np.repeat(f[None, :], ny, 0)

    full = np.ones((ny, nx))
    st = O.elastic_setup((nx, ny), (PER,) * 4, h, dt, rho * full, vp * full, vs * full, O.FP64, 0, P0=P0,
                         init={"sxx": rep(sxx), "syy": rep(lam / (lam + 2 * mu) * sxx), "vx": rep(vx)})
    _, E = st.run(10, energy=True)
    E = np.asarray(E) * 0.5 * h * P0 * P0 * dt / st.Z0
    return E[0] / (S * S * L * ny * h / (4.0 * (lam + 2.0 * mu))) - 1.0, float(np.ptp(E) / E[0])


def test_elastic_energy_in_physical_units_converges_to_continuous(oracle_lib):
    """The elastic discrete energy in physical units approaches the continuous
    strain energy of the standing P wave at second order and is conserved."""
    g64, d64 = _p_wave_energy_gap(64)
    g128, d128 = _p_wave_energy_gap(128)
    assert abs(g64) < 2e-3 and abs(g128) < abs(g64) / 3.0, (g64, g128)
    assert d64 <= 1e-12 and d128 <= 1e-12


def _vertical_p_pulse(top, ny=400, y0=100, width=6.0):
    """A plane P pulse (uniform in x, periodic x) of syy amplitude 1 at depth
    y0 in a homogeneous medium (rho = vp = h = 1, uniaxial strain: sxx =
    lambda / (lambda + 2 mu) syy), v = 0. It splits into an up- and a down-going
    pulse of amplitude 1/2. After 2 y0 / vp the up-going one has come back to
    y0 from the top face. Returns syy there then, and the largest |v_y| on the
    top row (in units of the incident 1 / (rho vp)) meanwhile."""
    nx = 8
    rho = np.ones((ny, nx))
    vp = np.ones((ny, nx))
    vs = vp / 1.73
    mu = rho * vs * vs
    lam = rho * vp * vp - 2.0 * mu
    dt = 0.5
    g = np.repeat(np.exp(-0.5 * ((np.arange(ny) - y0) / width) ** 2)[:, None], nx, 1)
    st = O.elastic_setup((nx, ny), (PER, PER, top, RIG), 1.0, dt, rho, vp, vs, O.FP64, 0,
                         init={"syy": g, "sxx": g * lam / (lam + 2.0 * mu)})
    vmax = 0.0
    for _ in range(int(round(2 * y0 / dt))):
        st.run(1)
        vmax = max(vmax, float(np.max(np.abs(st.f["vy"][0]))) / st.Z0)
    return float(st.f["syy"][y0, 0]), vmax


def test_free_surface_reflects_p_pulse_with_reversed_stress(oracle_lib):
    """Zero normal traction reflects a normally incident P wave with the
    stress reversed (reflection coefficient -1 for syy) and the particle
    velocity doubled at the surface; a rigid wall (zero normal velocity)
    reflects it with the stress unchanged and v_y near zero."""
    s_free, v_free = _vertical_p_pulse(FREE)
    s_rigid, v_rigid = _vertical_p_pulse(RIG)
    assert abs(s_free + 0.5) < 5e-3, s_free
    assert abs(s_rigid - 0.5) < 5e-3, s_rigid
    # incident v_y amplitude 1/2 (syy / (rho vp)); doubled on the surface
    assert abs(v_free - 1.0) < 5e-3, v_free
    assert v_rigid < 0.2, v_rigid


def _rayleigh_error(N, top=FREE, depth=4, cfl=0.5):
    """Largest relative L2 error over the five fields after one period of the
    analytic Rayleigh wave on a homogeneous half-space y >= 0 with a
    traction-free surface y = 0 (Poisson solid: vp = sqrt(3) vs; rho = vs = 1,
    wavelength L = 1 across a periodic x extent, N cells per wavelength, rigid
    bottom at 4 L where the wave has decayed to below 1e-4).
    Displacement potentials phi = A e^{-q y} e^{i(kx - wt)}, psi = B e^{-s y}
    e^{i(kx - wt)}, u_x = phi_x - psi_y, u_y = phi_y + psi_x, with
    q = k sqrt(1 - c^2/vp^2), s = k sqrt(1 - c^2/vs^2), the phase speed c the
    root of the Rayleigh equation (2 - c^2/vs^2)^2 = 4 sqrt(1 - c^2/vp^2)
    sqrt(1 - c^2/vs^2), and B fixed by sxy = 0 on the surface (syy = 0 there
    follows from the Rayleigh equation)."""
    L, rho0, beta = 1.0, 1.0, 1.0
    alpha = np.sqrt(3.0)
    h = L / N
    nx, ny = N, depth * N
    mu = rho0 * beta ** 2
    lam = rho0 * alpha ** 2 - 2.0 * mu
    f = lambda xi: (2 - xi) ** 2 - 4 * np.sqrt(1 - xi * beta ** 2 / alpha ** 2) * np.sqrt(1 - xi)
    xi = brentq(f, 0.5, 0.99)
    c = beta * np.sqrt(xi)
    k = 2 * np.pi / L
    w = c * k
    q = k * np.sqrt(1 - c ** 2 / alpha ** 2)
    s = k * np.sqrt(1 - c ** 2 / beta ** 2)
    A = 1.0
    B = -2j * k * q * A / (k * k * (2 - xi))

    def amp(y):
        eq, es = np.exp(-q * y), np.exp(-s * y)
        ux = 1j * k * A * eq + s * B * es
        uy = -q * A * eq + 1j * k * B * es
        return ux, uy, -1j * k * q * A * eq - s * s * B * es, q * q * A * eq - 1j * k * s * B * es

    def fields(ts, tv):
        xn, xh = np.arange(nx) * h, (np.arange(nx) + 0.5) * h
        yn, yh = np.arange(ny) * h, (np.arange(ny) + 0.5) * h
        ph = lambda x, t: np.exp(1j * (k * x[None, :] - w * t))
        ux, uy, dux, duy = amp(yn)
        exx, eyy = 1j * k * ux[:, None] * ph(xn, ts), duy[:, None] * ph(xn, ts)
        out = {"sxx": np.real((lam + 2 * mu) * exx + lam * eyy),
               "syy": np.real(lam * exx + (lam + 2 * mu) * eyy),
               "vx": np.real(-1j * w * ux[:, None] * ph(xh, tv))}
        ux, uy, dux, duy = amp(yh)
        out["vy"] = np.real(-1j * w * uy[:, None] * ph(xn, tv))
        out["sxy"] = np.real(mu * (dux[:, None] + 1j * k * uy[:, None]) * ph(xh, ts))
        return out

    dt = cfl * h / alpha
    n = int(round(L / c / dt))
    full = np.ones((ny, nx))
    st = O.elastic_setup((nx, ny), (PER, PER, top, RIG), h, dt, rho0 * full, alpha * full, beta * full,
                         O.FP64, 0, init=fields(0.0, -0.5 * dt))
    # the exact syy vanishes on the surface row, which the closure holds at zero
    st.run(n)
    ref = fields(n * dt, (n - 0.5) * dt)
    err = {}
    for name, r in ref.items():
        num = st.f[name] / st.Z0 if name in ("vx", "vy") else st.f[name]
        err[name] = np.linalg.norm(num - r) / np.linalg.norm(r)
    return max(err.values()), err


def test_free_surface_rayleigh_wave_converges(oracle_lib):
    """The Rayleigh wave is the free surface's own mode: its phase speed
    (0.9194 vs here) and its decay with depth are fixed by the two traction
    conditions, so a wrong image parity, a missing reduced modulus on the
    surface row or a rigid top gives an O(1) error. With the closure the error
    after one period falls at second order in h for the stresses and v_y
    (about 1.5 for v_x, whose surface row sits on the mirror plane)."""
    e32, d32 = _rayleigh_error(32)
    e64, d64 = _rayleigh_error(64)
    assert e64 < 7e-3, d64
    for name in ("sxx", "syy", "vy", "sxy"):
        assert d32[name] / d64[name] > 3.4, (name, d32[name], d64[name])
    assert d32["vx"] / d64["vx"] > 2.5, (d32["vx"], d64["vx"])
    e_rigid, _ = _rayleigh_error(32, top=RIG)
    assert e_rigid > 0.5, e_rigid
