"""Where the half-precision error comes from: an error split computed with the
CPU oracle only (the GPU path computes the same bits as the oracle's
emulation, which the parity tests check).

Each row runs one workload in a variant and reports the relative L2 error
against the binary64 scheme with unrounded coefficients (final pressure field,
or the receiver trace for W0) and the largest relative energy change. The
variants separate (Section 5, "Operator" and "Range"):
  * the rounding of the multipliers a and b to the storage format,
  * the rounding of the stencil weight 1/24,
  * the stencil's reading of the rounded stored value (half storage with the
    compensation carried, every operation and coefficient in binary64),
from the paper's method (half storage and arithmetic, plain or sum_3op), the
binary32-register variant, and a stencil that reads the stored pair V + T
(not the paper's scheme) with binary32 weight and multipliers.

Usage: python tests/accuracy_split.py [acoustic2d_256] [w0] [acoustic3d_recipe] [--small]
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import oracle as O  # noqa: E402
from paper_2310_00236_gb300 import inputs  # noqa: E402

F64, F32, F16 = O.FP64, O.FP32, O.FP16

VARIANTS = [
    ("binary64, a and b rounded to binary16", dict(store_fmt=F64, comp=0, coef_fmt=F16)),
    ("binary64, 1/24 rounded to binary16", dict(store_fmt=F64, comp=0, c2_fmt=F16)),
    ("binary64, a, b and 1/24 rounded to binary16", dict(store_fmt=F64, comp=0, coef_fmt=F16, c2_fmt=F16)),
    ("binary16 storage + compensation, all else binary64", dict(store_fmt=F16, comp=3, arith_fmt=F64,
                                                                stencil_fmt=F64, coef_fmt=F64)),
    ("fp16 plain (Algorithm 1)", dict(store_fmt=F16, comp=0)),
    ("fp16 + sum_3op (Algorithm 2)", dict(store_fmt=F16, comp=3)),
    ("fp16 storage, binary32 registers, compensated", dict(store_fmt=F16, comp=3, arith_fmt=F32)),
    ("fp16 pairs read by a binary32 stencil (not the paper)", dict(store_fmt=F16, comp=3, arith_fmt=F32,
                                                                   pair_stencil=True, coef_fmt=F32)),
    ("fp32", dict(store_fmt=F32, comp=0)),
]


def acoustic2d_256(small=False):
    """2D, rho = c = 1, p = 0 walls, centred Gaussian (sigma 0.05), CFL 0.5."""
    n, steps = (128, 1000) if small else (256, 2000)
    h = 1.0 / n
    x = np.arange(n) * h
    X, Y = np.meshgrid(x, x)
    return dict(name=f"2D acoustic {n}^2, CFL 0.5, {steps} steps", shape=(n, n), bc=(1, 1), h=h, dt=0.5 * h,
                rho=np.ones((n, n)), c=np.ones((n, n)),
                p0=np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / (2 * 0.05 ** 2)), steps=steps)


def w0(small=False):
    """The paper's regime (Section 5): periodic, rho = c = 1, h = 1/125,
    dt = 1e-4 (CFL 0.0125), Ricker 5 Hz pressure source, receiver trace. The
    full 600^2 x 60000-step experiment is reduced to n^2 with the source at
    (n/3, n/3) and the receiver at (2n/3, 2n/3), run until the direct arrival
    has passed."""
    n, steps = (150, 9000) if small else (300, 16000)
    h, dt = 1.0 / 125.0, 1e-4
    wav = inputs.ricker_table(steps, dt, 5.0)
    return dict(name=f"W0-like {n}^2, CFL 0.0125, {steps} steps", shape=(n, n), bc=(0, 0), h=h, dt=dt,
                rho=np.ones((n, n)), c=np.ones((n, n)), p0=None, steps=steps,
                src=(n // 3, n // 3, wav * 0.5 * h), rec=(2 * n // 3, 2 * n // 3))


def acoustic3d_recipe(small=False):
    """The 3D benchmark recipe on an n^3 sample (velocity filter width scaled
    by n / 512, the Gaussian initial pressure kept at 6 cells), p = 0 walls,
    CFL 0.4."""
    n, steps = (32, 100) if small else (64, 400)
    w = inputs.acoustic_3d_random(n=n, sigma_cells=16.0 * n / 512, ic_sigma_cells=6.0,
                                  smooth_dtype=np.float64)
    return dict(name=f"3D recipe {n}^3, CFL 0.4, {steps} steps", shape=w["shape"], bc=(1, 1, 1),
                h=w["h"], dt=w["dt"], rho=w["rho"], c=w["c"], p0=w["p0"], steps=steps)


def run(case, **kw):
    st = O.acoustic_setup(case["shape"], case["bc"], case["h"], case["dt"], case["rho"], case["c"],
                          kw.pop("store_fmt"), kw.pop("comp"), p0=case["p0"], **kw)
    rec = None
    if case.get("src"):
        i, j, wav = case["src"]
        st.src_index = i + case["shape"][0] * j
        st.src = O.scale_source(wav, st.Z0, 1.0, case["h"], 2, st.cfg.arith_fmt)
        rec = [case["rec"][0] + case["shape"][0] * case["rec"][1]]
    tr, E = st.run(case["steps"], rec_index=rec, energy=True)
    out = tr[:, 0] if rec else st.p.copy()
    q = int(0.8 / case["dt"]) if rec else 0          # W0: after the source has stopped
    Eq = E[q:] if E.size > q + 1 else E
    return out, float(np.max(np.abs(Eq - Eq[0])) / abs(Eq[0]))


def split(case):
    ref, d64 = run(case, store_fmt=F64, comp=0)
    rows = [("binary64 (reference)", 0.0, d64)]
    for name, kw in VARIANTS:
        out, drift = run(case, **dict(kw))
        rows.append((name, float(np.linalg.norm(out - ref) / np.linalg.norm(ref)), drift))
    return rows


def main(argv):
    small = "--small" in argv
    which = [a for a in argv if not a.startswith("--")] or ["acoustic2d_256", "w0", "acoustic3d_recipe"]
    for key in which:
        case = {"acoustic2d_256": acoustic2d_256, "w0": w0, "acoustic3d_recipe": acoustic3d_recipe}[key](small)
        t0 = time.time()
        rows = split(case)
        print(f"\n{case['name']} ({time.time() - t0:.0f} s, {O.set_threads()} threads)\n")
        print("| variant | rel L2 vs binary64 | energy drift |")
        print("|---|---|---|")
        for name, e, d in rows:
            print(f"| {name} | {e:.2e} | {d:.1e} |")


if __name__ == "__main__":
    main(sys.argv[1:])
