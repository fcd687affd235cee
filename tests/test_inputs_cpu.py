"""Pins for the seeded synthetic inputs (the workload recipes).

Each test checks a property the recipe states, computed independently of the
generator's own formula: extremes and layer values, the smoothing width
through the empirical autocorrelation of the filtered noise, the Ricker
wavelet's spectral peak, the geometry of shots and receivers, time steps
from the stated CFL numbers, and determinism of the seeds.
"""
import numpy as np

from paper_2310_00236_gb300 import inputs


def test_gaussian_peak_width_and_axis_order():
    h, sigma = 0.5, 3.0
    g = inputs.gaussian((16, 12, 10), h, sigma)
    assert g.shape == (10, 12, 16)                     # (z, y, x)
    assert g[5, 6, 8] == 1.0                           # the centre node N/2 on each axis
    off = int(sigma / h)                               # one sigma along x
    np.testing.assert_allclose(g[5, 6, 8 + off], np.exp(-0.5), rtol=1e-15)
    np.testing.assert_allclose(g[5, 6 - off, 8], np.exp(-0.5), rtol=1e-15)
    assert np.argmax(g) == np.ravel_multi_index((5, 6, 8), g.shape)


def test_smooth_random_field_range_seed_and_correlation_length():
    """Filtered white noise: the covariance of a Gaussian filter of width
    sigma is exp(-r^2 / (4 sigma^2)), so the correlation at lag 2 sigma is
    1/e; the affine rescaling to [lo, hi] does not change it."""
    sigma = 4.0
    f = inputs.smooth_random_field((256, 256), 3, sigma, 1500.0, 4500.0)
    np.testing.assert_allclose([f.min(), f.max()], [1500.0, 4500.0], rtol=1e-12)
    assert np.array_equal(f, inputs.smooth_random_field((256, 256), 3, sigma, 1500.0, 4500.0))
    assert not np.array_equal(f, inputs.smooth_random_field((256, 256), 4, sigma, 1500.0, 4500.0))
    d = f - f.mean()

    def corr(lag):   # periodic, along x and along y
        return 0.5 * (np.mean(d * np.roll(d, lag, 1)) + np.mean(d * np.roll(d, lag, 0))) / np.mean(d * d)

    assert abs(corr(int(2 * sigma)) - np.exp(-1.0)) < 0.08
    assert abs(corr(int(sigma)) - np.exp(-0.25)) < 0.05
    assert abs(corr(int(4 * sigma))) < 0.1


def test_ricker_peak_zeros_and_spectrum():
    f0, t0 = 10.0, 0.12
    assert inputs.ricker(np.array([t0]), f0, t0)[0] == 1.0
    tz = t0 + 1.0 / (np.sqrt(2.0) * np.pi * f0)        # zero crossing of 1 - 2 (pi f tau)^2
    assert abs(inputs.ricker(np.array([tz]), f0, t0)[0]) < 1e-15
    dt = 1e-4
    w = inputs.ricker(np.arange(40000) * dt, f0, t0)   # 4 s, 0.25 Hz bins
    spec = np.abs(np.fft.rfft(w))
    fpk = np.fft.rfftfreq(w.size, dt)[np.argmax(spec)]
    assert abs(fpk - f0) <= 0.25                       # amplitude spectrum peaks at f0
    tab = inputs.ricker_table(8, 0.01, f0)             # pressure sources: t = (n + 1/2) dt
    np.testing.assert_array_equal(tab, inputs.ricker((np.arange(8) + 0.5) * 0.01, f0, 1.2 / f0))
    cut = inputs.ricker_table(100, 0.01, f0, t0=0.1, half_step=False, cutoff=0.5)
    assert np.all(cut[51:] == 0.0) and cut[50] != 0.0


def test_acoustic_3d_random_recipe():
    n = 32
    w = inputs.acoustic_3d_random(n=n, sigma_cells=2.0, ic_sigma_cells=3.0, smooth_dtype=np.float64)
    assert w["shape"] == (n, n, n) and w["c"].shape == (n, n, n)
    np.testing.assert_allclose([w["c"].min(), w["c"].max()], [1500.0, 4500.0], rtol=1e-12)
    assert np.all(w["rho"] == 1000.0)
    assert abs(w["dt"] * 4500.0 / w["h"] - 0.4) < 1e-15  # CFL 0.4 on the largest speed
    p0 = w["p0"]
    assert p0[n // 2, n // 2, n // 2] == 1.0
    np.testing.assert_allclose(p0[n // 2, n // 2, n // 2 + 3], np.exp(-0.5), rtol=1e-14)


def test_acoustic_3d_adjoint_geometry():
    n = 64
    w = inputs.acoustic_3d_adjoint(n=n, steps=50)
    shots, recs = np.array(w["shots"]), np.array(w["receivers"])
    assert shots.shape == (16, 3) and recs.shape == (64, 3)
    assert np.all(shots[:, 2] == 2) and np.all(recs[:, 2] == 2)    # depth index 2
    assert len({tuple(s) for s in shots}) == 16 and len({tuple(r) for r in recs}) == 64
    assert sorted(set(shots[:, 0])) == [8, 24, 40, 56]               # 4 x 4, cell centres
    assert sorted(set(recs[:, 1])) == [4, 12, 20, 28, 36, 44, 52, 60]  # 8 x 8
    assert w["c0"].min() >= 1500.0 and w["c0"].max() <= 4500.0
    # the start model is smoother than the true model
    def rough(c):
        return np.mean(np.abs(np.diff(c, axis=2)))
    assert rough(w["c0"]) < 0.5 * rough(w["c_true"])


def test_batch_shot_sides_and_shots():
    sides = inputs.shot_sides()
    assert sides.shape == (64,) and sides.min() >= 256 and sides.max() <= 2048
    assert int(np.sum(sides.astype(np.int64) ** 2)) == 98978600       # the batch's cells
    assert np.array_equal(sides, inputs.shot_sides())
    s = inputs.acoustic_2d_shot(5, 300, steps=40)
    assert s["shape"] == (300, 300) and s["src_idx"] == [150, 8]
    np.testing.assert_allclose([s["c"].min(), s["c"].max()], [1500.0, 4500.0], rtol=1e-12)
    assert abs(s["dt"] * 4500.0 / s["h"] - 0.4) < 1e-15


def test_elastic_layered_recipe():
    n = 60
    w = inputs.elastic_2d_layered(n=n, steps=400)
    vp, rho = w["vp"], w["rho"]
    for ys, v, r in ((range(0, 20), 2000.0, 2000.0), (range(20, 40), 3000.0, 2300.0),
                     (range(40, 60), 4000.0, 2600.0)):
        assert np.all(vp[list(ys)] == v) and np.all(rho[list(ys)] == r)
    np.testing.assert_array_equal(w["vs"], vp / 1.73)
    assert w["dt"] == 0.5 * 3.0 / 4000.0
    assert w["src_idx"] == (30, 10)
    ts = np.arange(400) * w["dt"]
    assert np.all(w["wavelet"][ts > 0.1] == 0.0)
    assert w["src_steps"] == int(round(0.1 / w["dt"]))
    k = int(np.argmax(np.abs(w["wavelet"])))                     # the peak at t0 = 0.05 s
    assert abs(ts[k] - 0.05) <= w["dt"]


def test_w0_paper_replica_recipe():
    w = inputs.acoustic_2d_w0(steps=10)
    assert w["shape"] == (600, 600) and w["h"] == 1.0 / 125.0 and w["dt"] == 1e-4
    assert abs(1.0 * w["dt"] / w["h"] - 0.0125) < 1e-15                # CFL with c = 1
    assert abs(1.0 / (2.5 * 5.0) / w["h"] - 10.0) < 1e-12              # 10 points per wavelength at 2.5 f0
    assert w["src_idx"] == [200, 200] and w["rec_idx"] == [400, 400]
    assert inputs.acoustic_2d_w0()["steps"] == 60000
    w3 = inputs.acoustic_2d_w0(refine=3, steps=10)
    assert w3["shape"] == (1800, 1800) and w3["src_idx"] == [600, 600]
    assert abs(w3["h"] * 3 - w["h"]) < 1e-18 and abs(w3["dt"] * 3 - w["dt"]) < 1e-18
