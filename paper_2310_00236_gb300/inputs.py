"""Seeded synthetic inputs for the wave workloads.

This module only draws and shapes input data (materials, initial fields,
source wavelets). It holds none of the scheme's arithmetic, so both the CUDA
path and the CPU oracle can be fed from it without sharing any of the method.

Array convention: numpy float64, shaped (z, y, x) in 3D and (y, x) in 2D,
x fastest. Along each axis with N cells and spacing h, p nodes sit at m*h for
m = 0..N-1 (the node at N*h is the far wall, or node 0 again when periodic).
"""
from __future__ import annotations

import numpy as np


def node_coords(n: int, h: float) -> np.ndarray:
    return np.arange(n, dtype=np.float64) * h


def gaussian(shape, h: float, sigma: float, center=None, peak: float = 1.0) -> np.ndarray:
    """Gaussian bump exp(-|x - xc|^2 / (2 sigma^2)) sampled on p nodes.

    shape: cells per axis in (x, y[, z]) order; the result is reversed to
    (z, y, x). The default centre is the domain centre, node N/2 on each axis.
    """
    nd = len(shape)
    if center is None:
        center = [0.5 * shape[a] * h for a in range(nd)]
    # separable: the product of one 1D Gaussian per axis, outermost axis first
    out = np.full((), peak, dtype=np.float64)
    for a in reversed(range(nd)):
        x = node_coords(shape[a], h) - center[a]
        g = np.exp(-(x * x) / (2.0 * sigma * sigma))
        out = np.multiply.outer(out, g)
    return np.ascontiguousarray(out)


def smooth_random_field(shape, seed: int, sigma_cells: float, lo: float, hi: float,
                        dtype=np.float64) -> np.ndarray:
    """Gaussian-filtered white noise (periodic FFT filter), affinely rescaled
    to [lo, hi]. shape in (x, y[, z]) order; result (z, y, x).

    The noise is numpy's PCG64 standard normal with the given seed, drawn in
    (z, y, x) order.
    """
    try:
        import scipy.fft as sfft
        rfftn = lambda a: sfft.rfftn(a, workers=-1)
        irfftn = lambda a, s: sfft.irfftn(a, s=s, workers=-1)
    except ImportError:
        rfftn = np.fft.rfftn
        irfftn = lambda a, s: np.fft.irfftn(a, s=s, axes=tuple(range(len(s))))
    rshape = tuple(shape[::-1])
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(rshape, dtype=np.float32 if dtype == np.float32 else np.float64)
    spec = rfftn(noise)
    del noise
    kernel = None
    for ax, n in enumerate(rshape):
        if ax == len(rshape) - 1:
            k = np.fft.rfftfreq(n)
        else:
            k = np.fft.fftfreq(n)
        g = np.exp(-2.0 * (np.pi * sigma_cells * k) ** 2)
        shp = [1] * len(rshape)
        shp[ax] = g.size
        g = g.reshape(shp)
        kernel = g if kernel is None else kernel * g
    spec *= kernel.astype(spec.real.dtype)
    field = irfftn(spec, rshape)
    del spec
    fmin, fmax = float(field.min()), float(field.max())
    field = lo + (field - fmin) * ((hi - lo) / (fmax - fmin))
    return np.ascontiguousarray(field.astype(np.float64))


def ricker(t: np.ndarray, f: float, t0: float) -> np.ndarray:
    """Ricker wavelet (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2), tau = t - t0."""
    tau = np.asarray(t, dtype=np.float64) - t0
    a = (np.pi * f * tau) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def ricker_table(nt: int, dt: float, f: float, t0: float | None = None,
                 half_step: bool = True, cutoff: float | None = None) -> np.ndarray:
    """Wavelet samples for steps 0..nt-1 at t = (n + 1/2) dt (pressure
    sources) or t = n dt; t0 defaults to 1.2 / f. Samples after `cutoff`
    seconds are zero."""
    if t0 is None:
        t0 = 1.2 / f
    t = (np.arange(nt, dtype=np.float64) + (0.5 if half_step else 0.0)) * dt
    w = ricker(t, f, t0)
    if cutoff is not None:
        w[t > cutoff] = 0.0
    return w


# ---------------------------------------------------------------------------
# Workload recipes (sizes and value distributions of the benchmark configs)
# ---------------------------------------------------------------------------

def acoustic_2d_gaussian(n: int = 256, steps: int = 2000, cfl: float = 0.5, sigma: float = 0.05):
    """2D acoustic, n x n cells on [0,1]^2, h = 1/n, rho = c = 1, p = 0 walls,
    centred Gaussian initial pressure, v = 0, dt = cfl * h."""
    h = 1.0 / n
    return dict(ndim=2, shape=(n, n), h=h, dt=cfl * h, steps=steps,
                rho=np.ones((n, n)), c=np.ones((n, n)),
                p0=gaussian((n, n), h, sigma), P0=1.0)


def acoustic_3d_random(n: int = 512, steps: int = 1000, cfl: float = 0.4, h: float = 10.0,
                       seed: int = 0, sigma_cells: float = 16.0, vmin: float = 1500.0,
                       vmax: float = 4500.0, rho: float = 1000.0, ic_sigma_cells: float = 6.0,
                       smooth_dtype=np.float32):
    """3D acoustic, n^3 cells, spacing h metres, density rho, smooth random
    velocity in [vmin, vmax] (seeded Gaussian-filtered noise), p = 0 walls,
    Gaussian initial pressure of width ic_sigma_cells * h and peak 1 Pa,
    dt = cfl * h / vmax."""
    shape = (n, n, n)
    c = smooth_random_field(shape, seed, sigma_cells, vmin, vmax, dtype=smooth_dtype)
    return dict(ndim=3, shape=shape, h=h, dt=cfl * h / vmax, steps=steps,
                rho=np.full(c.shape, rho), c=c,
                p0=gaussian(shape, h, ic_sigma_cells * h), P0=1.0)


def gaussian_smooth(field: np.ndarray, sigma_cells: float) -> np.ndarray:
    """Periodic Gaussian filter of a (z, y, x) or (y, x) array (FFT), the same
    kernel smooth_random_field applies to its noise."""
    spec = np.fft.rfftn(field)
    shp = field.shape
    for ax, n in enumerate(shp):
        k = np.fft.rfftfreq(n) if ax == len(shp) - 1 else np.fft.fftfreq(n)
        g = np.exp(-2.0 * (np.pi * sigma_cells * k) ** 2)
        s = [1] * len(shp)
        s[ax] = g.size
        spec *= g.reshape(s)
    return np.ascontiguousarray(np.fft.irfftn(spec, s=shp, axes=tuple(range(len(shp)))))


def acoustic_3d_adjoint(n: int = 256, steps: int = 1500, h: float = 10.0, cfl: float = 0.4,
                        f0: float = 10.0, rho: float = 1000.0, vmin: float = 1500.0,
                        vmax: float = 4500.0, start_sigma_cells: float = 32.0):
    """3D acoustic inversion experiment: the smooth random velocity of
    acoustic_3d_random (seed 0, filter width 16 n / 512 cells) as the true
    model, the true model Gaussian-filtered with start_sigma_cells as the
    start model, constant density, rigid walls, 16 shots on a 4 x 4 grid and 64
    receivers on an 8 x 8 grid, both at depth index 2 (z), Ricker f0 sources,
    dt = cfl h / vmax. Index tuples are (i, j, k)."""
    shape = (n, n, n)
    c_true = smooth_random_field(shape, 0, 16.0 * n / 512, vmin, vmax)
    c0 = np.clip(gaussian_smooth(c_true, start_sigma_cells), vmin, vmax)
    dt = cfl * h / vmax
    shots = [(int(n * (a + 0.5) / 4), int(n * (b + 0.5) / 4), 2) for b in range(4) for a in range(4)]
    recs = [(int(n * (a + 0.5) / 8), int(n * (b + 0.5) / 8), 2) for b in range(8) for a in range(8)]
    return dict(ndim=3, shape=shape, h=h, dt=dt, steps=steps, rho=np.full(c_true.shape, rho),
                c_true=c_true, c0=np.ascontiguousarray(c0), shots=shots, receivers=recs,
                wavelet=ricker_table(steps, dt, f0), P0=1.0, z0=rho * vmax)


def acoustic_2d_w0(refine: int = 1, f0: float = 5.0, steps: int | None = None):
    """The paper's acoustic accuracy experiment (Section 5): 600 x 600 cells of
    h = 1/125 m (10 points per wavelength), rho = c = 1, periodic, dt = 1e-4 s
    (CFL 0.0125), 60000 steps, Ricker f0 pressure source at node (200, 200),
    receiver at node (400, 400). refine = 3 gives the 30-points-per-wavelength
    grid of the same domain (h / 3, dt / 3, three times the steps, nodes x 3)."""
    r = int(refine)
    n = 600 * r
    h = 1.0 / (125.0 * r)
    dt = 1e-4 / r
    nsteps = 60000 * r if steps is None else steps
    return dict(ndim=2, shape=(n, n), h=h, dt=dt, steps=nsteps, rho=np.ones((n, n)), c=np.ones((n, n)),
                src_idx=[200 * r, 200 * r], rec_idx=[400 * r, 400 * r],
                wavelet=ricker_table(nsteps, dt, f0), refine=r)


def shot_sides(nshots: int = 64, seed: int = 1, lo: int = 256, hi: int = 2048) -> np.ndarray:
    """Grid sides of a batch of 2D shots: uniform integers in [lo, hi] from
    numpy's PCG64 with the given seed."""
    return np.random.default_rng(seed).integers(lo, hi + 1, nshots)


def acoustic_2d_shot(i: int, side: int, steps: int = 3000, h: float = 10.0, cfl: float = 0.4,
                     f0: float = 10.0, rho: float = 1000.0, vmin: float = 1500.0,
                     vmax: float = 4500.0):
    """Shot i of a batch: side x side cells, spacing h, its own smooth random
    velocity (seed 100 + i, filter width side/32 cells, rescaled to
    [vmin, vmax]), constant density, rigid walls, a Ricker f0 pressure source
    at node (side/2, 8), dt = cfl h / vmax (the same for every shot)."""
    c = smooth_random_field((side, side), 100 + i, side / 32.0, vmin, vmax)
    dt = cfl * h / vmax
    return dict(ndim=2, shape=(side, side), h=h, dt=dt, steps=steps,
                rho=np.full(c.shape, rho), c=c, src_idx=[side // 2, 8],
                wavelet=ricker_table(steps, dt, f0), P0=1e5, z0=rho * vmax)


def elastic_2d_layered(n: int = 1024, steps: int = 4000, h: float = 3.0, f0: float = 15.0,
                       cutoff: float = 0.1):
    """2D isotropic elastic, n x n cells, spacing h: three horizontal layers
    y in [0, n/3), [n/3, 2n/3), [2n/3, n) with Vp 2000 / 3000 / 4000 m/s,
    Vs = Vp / 1.73, rho 2000 / 2300 / 2600 kg/m^3; free top, rigid other
    sides; Ricker f0 vertical force at (n/2, 10) for `cutoff` seconds (t0 = cutoff/2,
    sampled at t_n) then source-free; dt = 0.5 h / 4000."""
    y = np.arange(n)
    vp1 = np.where(y < n // 3, 2000.0, np.where(y < 2 * n // 3, 3000.0, 4000.0))
    rho1 = np.where(y < n // 3, 2000.0, np.where(y < 2 * n // 3, 2300.0, 2600.0))
    vp = np.ascontiguousarray(np.repeat(vp1[:, None], n, 1))
    rho = np.ascontiguousarray(np.repeat(rho1[:, None], n, 1))
    dt = 0.5 * h / 4000.0
    wav = ricker_table(steps, dt, f0, t0=0.5 * cutoff, half_step=False, cutoff=cutoff)
    return dict(ndim=2, shape=(n, n), h=h, dt=dt, steps=steps, rho=rho, vp=vp, vs=vp / 1.73,
                src_idx=(n // 2, 10), wavelet=wav, src_steps=int(round(cutoff / dt)))
