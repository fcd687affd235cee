"""The paper's qualitative findings, as assertions on the oracle.

The figures are not available, so each statement of the text becomes a
measurable check on a scaled-down version of the paper's regime (small CFL,
about ten points per wavelength, periodic walls, Section 3):

1. fp16 with the plain update loses energy (Section 3, text after Figs 8-11).
2. fp16 with sum_3op keeps the energy and agrees with fp64 to about the
   discretisation error (Section 4, text after Figs 12-16).
3. Promoting only the stencil to fp64 does not cure the plain update; adding
   compensation does (Appendix B).
4. sum_3op and sum_6op give very similar results (Section 4; Appendix A).

A mistake in the compensated update (a dropped carry, a wrong sign, the carry
added in the wrong place) makes 2-4 fail.
"""
import numpy as np
import pytest

import oracle as O
from paper_2310_00236_gb300 import inputs

N = 64
CFL = 0.0125        # the paper's dt = 1e-4 s with h = 1/125 m and c = 1 m/s
STEPS = 4000


def _pulse(fmt, comp, stencil_fmt=None):
    h = 1.0 / N
    p0 = inputs.gaussian((N, N), h, 3.0 * h)
    st = O.acoustic_setup((N, N), (O.BC_PERIODIC,) * 2, h, CFL * h, np.ones((N, N)),
                          np.ones((N, N)), fmt, comp, stencil_fmt=stencil_fmt, p0=p0)
    _, E = st.run(STEPS, energy=True)
    return st.p.copy(), (E - E[0]) / E[0]


@pytest.fixture(scope="module")
def runs(oracle_lib):
    return {
        "fp64": _pulse(O.FP64, 0),
        "fp16": _pulse(O.FP16, 0),
        "fp16_3op": _pulse(O.FP16, 3),
        "fp16_6op": _pulse(O.FP16, 6),
        "fp16_stencil64": _pulse(O.FP16, 0, O.FP64),
        "fp16_stencil64_3op": _pulse(O.FP16, 3, O.FP64),
    }


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_fp16_plain_update_loses_energy(runs):
    _, dE = runs["fp16"]
    quarters = dE[[STEPS // 4, STEPS // 2, 3 * STEPS // 4, STEPS - 1]]
    assert np.all(np.diff(quarters) < 0)          # monotone loss
    assert dE[-1] < -0.01


def test_fp16_compensated_keeps_energy_and_accuracy(runs):
    _, dE3 = runs["fp16_3op"]
    loss = -runs["fp16"][1][-1]
    assert np.max(np.abs(dE3)) < 0.02 * loss
    p64 = runs["fp64"][0]
    assert _rel(runs["fp16_3op"][0], p64) < 0.2 * _rel(runs["fp16"][0], p64)


def test_stencil_promotion_alone_does_not_help(runs):
    _, dE = runs["fp16_stencil64"]
    assert dE[-1] < -0.01
    _, dEc = runs["fp16_stencil64_3op"]
    assert np.max(np.abs(dEc)) < 0.02 * -dE[-1]


def test_3op_and_6op_are_close(runs):
    p3, p6, p0 = runs["fp16_3op"][0], runs["fp16_6op"][0], runs["fp16"][0]
    assert np.linalg.norm(p3 - p6) <= 0.1 * np.linalg.norm(p0 - p3)


def test_compensated_error_at_the_level_of_discretisation_error(oracle_lib):
    """Periodic plane standing wave with ten points per wavelength, one domain
    crossing at the paper's CFL: the fp16 + sum_3op deviation from fp64 is of
    the order of fp64's own discretisation error (distance to the exact
    solution); the plain fp16 deviation is an order of magnitude larger."""
    n = 40
    h = 1.0 / n
    dt = CFL * h
    k = 2 * np.pi * 4
    x = np.arange(n) * h
    X, _ = np.meshgrid(x, x, indexing="xy")
    Xh, _ = np.meshgrid(x + 0.5 * h, x, indexing="xy")
    p0 = np.cos(k * X)
    vx = np.sin(k * -0.5 * dt) / k * (-k) * np.sin(k * Xh)
    steps = int(round(1.0 / dt))
    out = {}
    for name, (fmt, comp) in {"fp64": (O.FP64, 0), "fp16": (O.FP16, 0),
                              "fp16_3op": (O.FP16, 3)}.items():
        st = O.acoustic_setup((n, n), (O.BC_PERIODIC,) * 2, h, dt, np.ones((n, n)),
                              np.ones((n, n)), fmt, comp, p0=p0, v0=[vx, np.zeros_like(vx)])
        st.run(steps)
        out[name] = st.p
    exact = np.cos(k * steps * dt) * p0
    disc = _rel(out["fp64"], exact)
    assert _rel(out["fp16_3op"], out["fp64"]) < 3.0 * disc
    assert _rel(out["fp16"], out["fp64"]) > 10.0 * disc
