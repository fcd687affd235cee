"""The paper's acoustic accuracy experiment (Section 5: 600 x 600 periodic
grid, 10 points per wavelength, rho = c = 1, CFL 0.0125, 60000 steps, Ricker
source, one receiver) on the GPU path, with the paper's qualitative claims as
assertions:

* plain binary16 ends with less energy than it had when the source stopped
  (here -2.2 %; the decrease is not monotone on this grid: the energy first
  rises by several per cent, then falls), while the compensated update keeps
  the energy change at least ten times smaller;
* the compensated update cuts the receiver-trace error against the binary32
  run several fold;
* sum_3op and sum_6op give the same result here (the stored value always
  dominates the increment), far closer to each other than to the plain run.

The paper's further claim that the compensated binary16 trace error stays
below the gap between the 10- and 30-points-per-wavelength binary64 runs is
not asserted: on this path the error is 3.4e-2 against a gap of 7.8e-3 (the
rounding of the stored stencil inputs, which compensation does not repair);
the figures come from `bench.py --leg w0`. It does hold for the pair
precision (binary16 V and T, stencil taps RN32(V + T), binary32
multipliers; not the paper's scheme) once the field is scaled into the
normal range of binary16 (P0 = 1/64, Section 5 "Range"): 2.6e-4 against the
binary32 run, asserted below.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(W, prec, comp, field_scale=1.0):
    import torch
    from paper_2310_00236_gb300 import inputs
    w = inputs.acoustic_2d_w0(1)
    n = w["steps"]
    ctx = W.wave_create(w["shape"], w["h"], w["rho"], w["c"], w["dt"], prec, comp,
                        bc=[W.WAVE_BC_PERIODIC] * 4 + [0, 0], field_scale=field_scale)
    try:
        W.wave_set_source(ctx, W.WAVE_F_P, w["src_idx"], w["wavelet"] * (0.5 / 125.0))
        tr = torch.zeros((n, 1), dtype=torch.float32, device="cuda")
        W.wave_set_receivers(ctx, W.WAVE_F_P, [w["rec_idx"]], tr, n)
        en = torch.zeros(n, dtype=torch.float64, device="cuda")
        W.wave_set_energy_trace(ctx, en, n)
        W.wave_step(ctx, n)
        torch.cuda.synchronize()
        # traces sample the stored (scaled) field
        return tr.cpu().numpy()[:, 0].astype(np.float64) * field_scale, en.cpu().numpy(), int(0.8 / w["dt"])
    finally:
        W.wave_destroy(ctx)


def test_w0_paper_claims_on_gpu():
    from paper_2310_00236_gb300 import wave as W
    ref, e32, quiet = _run(W, W.WAVE_FP32, 0)
    naive, e_n, _ = _run(W, W.WAVE_FP16, 0)
    k3, e_3, _ = _run(W, W.WAVE_FP16, 3)
    k6, e_6, _ = _run(W, W.WAVE_FP16, 6)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    drift = lambda e: (e[-1] - e[quiet]) / e[quiet]
    # energy: binary32 holds it, plain binary16 loses it, compensation keeps it
    assert abs(drift(e32)) < 1e-5
    assert drift(e_n) < -5e-3
    assert abs(drift(e_3)) * 10 < abs(drift(e_n))
    # trace error against binary32
    assert rel(k3, ref) * 4 < rel(naive, ref)
    assert rel(k6, k3) <= 0.1 * rel(naive, k3)


def test_w0_pair_precision_scaled_meets_the_discretisation_gap():
    """The pair precision with P0 = 1/64: the receiver trace within 1e-3 of
    the binary32 run (the 10- vs 30-point gap is 7.8e-3) and ten times closer
    than fp16 + sum_3op at the same scaling; the energy change after the
    source far below plain binary16's."""
    from paper_2310_00236_gb300 import wave as W
    ref, _, quiet = _run(W, W.WAVE_FP32, 0)
    pairs, e_p, _ = _run(W, W.WAVE_FP16_PAIRS, 3, field_scale=1.0 / 64)
    k3, _, _ = _run(W, W.WAVE_FP16, 3, field_scale=1.0 / 64)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    assert rel(pairs, ref) < 1e-3, rel(pairs, ref)
    assert rel(pairs, ref) * 10 < rel(k3, ref)
    assert abs((e_p[-1] - e_p[quiet]) / e_p[quiet]) < 1e-4
