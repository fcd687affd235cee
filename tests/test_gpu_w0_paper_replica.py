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
the figures come from `bench.py --leg w0`.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(W, prec, comp):
    import torch
    from paper_2310_00236_gb300 import inputs
    w = inputs.acoustic_2d_w0(1)
    n = w["steps"]
    ctx = W.wave_create(w["shape"], w["h"], w["rho"], w["c"], w["dt"], prec, comp,
                        bc=[W.WAVE_BC_PERIODIC] * 4 + [0, 0])
    try:
        W.wave_set_source(ctx, W.WAVE_F_P, w["src_idx"], w["wavelet"] * (0.5 / 125.0))
        tr = torch.zeros((n, 1), dtype=torch.float32, device="cuda")
        W.wave_set_receivers(ctx, W.WAVE_F_P, [w["rec_idx"]], tr, n)
        en = torch.zeros(n, dtype=torch.float64, device="cuda")
        W.wave_set_energy_trace(ctx, en, n)
        W.wave_step(ctx, n)
        torch.cuda.synchronize()
        return tr.cpu().numpy()[:, 0].astype(np.float64), en.cpu().numpy(), int(0.8 / w["dt"])
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
