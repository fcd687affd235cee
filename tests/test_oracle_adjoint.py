"""Pins of the oracle's discrete adjoint (reverse-mode gradient of the binary64
acoustic scheme), independent of its own reverse sweep:

* the dot-product identity <F x, y> = <x, F^T y> for the linear map F from the
  initial pressure to the recorded pressure traces (no source), with F applied
  by the forward solver and F^T by the adjoint sweep, on periodic and rigid
  grids in 2D and 3D, receivers everywhere on the smallest grid;
* central finite differences of the misfit J(c) = 1/2 |traces(c) - d_obs|^2,
  each J evaluated by the forward solver alone, against <dJ/dc, dc> for smooth
  model perturbations dc, with a source and a varying density.
"""
import numpy as np
import pytest

import oracle as O
from paper_2310_00236_gb300 import inputs

R, P = O.BC_RIGID, O.BC_PERIODIC


def _model(shape, seed):
    c = inputs.smooth_random_field(shape, seed, 2.0, 1500.0, 4500.0)
    rho = 1000.0 + 200.0 * inputs.smooth_random_field(shape, seed + 7, 2.0, -1.0, 1.0)
    return rho, c


def _state(shape, bc, rho, c, h=10.0, cfl=0.4, p0=None, src=None):
    dt = cfl * h / 4500.0
    st = O.acoustic_setup(shape, bc, h, dt, rho, c, O.FP64, 0, P0=1.0, p0=p0)
    if src is not None:
        idx, wav = src
        st.src_index = int(np.ravel_multi_index(tuple(idx[::-1]), st.shape))
        st.src = O.scale_source(wav, st.Z0, 1.0, h, len(shape), O.FP64)
    return st


@pytest.mark.parametrize("shape,bc,nsteps", [((8, 8), (R, R), 30), ((8, 8), (P, R), 30),
                                             ((24, 20), (R, P), 60), ((12, 10, 8), (R, R, R), 25),
                                             ((10, 8, 9), (P, R, P), 25)])
def test_adjoint_dot_product_identity(shape, bc, nsteps):
    rng = np.random.default_rng(sum(shape))
    rho, c = _model(shape, 3)
    st = _state(shape, bc, rho, c)
    npts = int(np.prod(shape))
    x = rng.standard_normal(st.shape)
    if npts <= 64:
        rec = np.arange(npts)
    else:
        rec = rng.choice(npts, 12, replace=False)
    y = rng.standard_normal((nsteps, len(rec)))
    fwd = st.copy()
    fwd.p = x.copy()
    Fx, _ = fwd.run(nsteps, 0, rec)
    st.p = x.copy()
    out = O.acoustic_adjoint(st, c, nsteps, rec, residual=y)
    assert np.array_equal(out["traces"], Fx)
    lhs = float(np.sum(Fx * y))
    rhs = float(np.sum(x * out["p0_bar"]))
    scale = float(np.sum(np.abs(Fx * y)))
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs, scale)


def _misfit(shape, bc, rho, c, nsteps, rec, d_obs, p0, src):
    st = _state(shape, bc, rho, c, p0=p0, src=src)
    tr, _ = st.run(nsteps, 0, rec)
    return 0.5 * float(np.sum((tr - d_obs) ** 2))


@pytest.mark.parametrize("shape,bc,nsteps", [((32, 24), (R, R), 120), ((20, 16), (P, R), 80),
                                             ((12, 12, 10), (R, R, R), 40)])
def test_adjoint_gradient_matches_central_differences(shape, bc, nsteps):
    nd = len(shape)
    rho, c_true = _model(shape, 11)
    c = c_true.copy()
    c[tuple(s // 2 for s in c.shape)] *= 1.0  # start model = true model, then smoothed away
    c = 0.7 * c_true + 0.3 * inputs.smooth_random_field(shape, 12, 4.0, 1500.0, 4500.0)
    h, cfl = 10.0, 0.4
    dt = cfl * h / 4500.0
    wav = inputs.ricker_table(nsteps, dt, 1.0 / (25 * dt))
    src = ([s // 2 for s in shape[:-1]] + [2], wav * 1e3)
    p0 = None
    rng = np.random.default_rng(5)
    npts = int(np.prod(shape))
    rec = rng.choice(npts, 10, replace=False)
    truth = _state(shape, bc, rho, c_true, p0=p0, src=src)
    d_obs, _ = truth.run(nsteps, 0, rec)
    st = _state(shape, bc, rho, c, p0=p0, src=src)
    out = O.acoustic_adjoint(st, c, nsteps, rec, d_obs=d_obs)
    J0 = _misfit(shape, bc, rho, c, nsteps, rec, d_obs, p0, src)
    assert out["J"] == pytest.approx(J0, rel=1e-13)
    assert J0 > 0
    for seed in (21, 22):
        dc = inputs.smooth_random_field(shape, seed, 2.0, -50.0, 50.0)
        eps = 1e-3
        Jp = _misfit(shape, bc, rho, c + eps * dc, nsteps, rec, d_obs, p0, src)
        Jm = _misfit(shape, bc, rho, c - eps * dc, nsteps, rec, d_obs, p0, src)
        fd = (Jp - Jm) / (2 * eps)
        an = float(np.sum(out["grad_c"] * dc))
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an, nd)


def test_adjoint_rejects_half_precision_state():
    shape = (8, 8)
    rho, c = _model(shape, 1)
    st = O.acoustic_setup(shape, (R, R), 10.0, 0.4 * 10 / 4500, rho, c, O.FP16, 3, P0=1.0)
    with pytest.raises(ValueError):
        O.acoustic_adjoint(st, c, 4, [3], residual=np.ones((4, 1)))
