"""Brute-force pins of the oracle's spatial operators on tiny grids.

The oracle's gradient (p -> v) and divergence (v -> p) maps are extracted from
single impulses and compared with dense matrices assembled here, independently,
from the stencil weights printed in Section 3 (tests/golden/stencil_weights.txt)
and the boundary rules (wrap-around, or the odd/even images that keep p = 0 on
rigid walls). Then the structural facts are checked: the gradient is exactly
minus the transpose of the divergence (the skew structure that makes the
discrete energy conserved), and the leapfrog amplification matrix has all its
eigenvalues on the unit circle below the stability limit and not above it.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _weights():
    w = {}
    with open(os.path.join(GOLDEN, "stencil_weights.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            off, wt = line.split()
            w[float(off)] = float(Fraction(wt))
    return w


def _ext_1d(N, bc, node):
    """Dense map from the N stored values to positions -3..N+2 along one axis:
    row r corresponds to position m = r - 3 (node m, or half point m + 1/2)."""
    E = np.zeros((N + 6, N))
    for r in range(N + 6):
        m = r - 3
        if 0 <= m < N:
            E[r, m] = 1.0
        elif bc == O.BC_PERIODIC:
            E[r, m % N] = 1.0
        elif node:  # odd about nodes 0 and N, zero at N
            if m < 0:
                E[r, -m] = -1.0
            elif m > N:
                E[r, 2 * N - m] = -1.0
        else:  # half points: even about the walls
            E[r, (-1 - m) if m < 0 else (2 * N - 1 - m)] = 1.0
    return E


def _diff_1d(N, bc, to_half):
    """Undivided 4th-order staggered derivative along one axis.
    to_half: node field -> half points (gradient); else half -> nodes."""
    w = _weights()
    E = _ext_1d(N, bc, node=to_half)
    D = np.zeros((N, N))
    for m in range(N):
        if to_half:   # target m+1/2: nodes m-1, m, m+1, m+2 at offsets -3/2..3/2
            taps = {m - 1: w[-1.5], m: w[-0.5], m + 1: w[0.5], m + 2: w[1.5]}
        else:         # target node m: half points m-2, m-1, m, m+1 (+1/2)
            taps = {m - 2: w[-1.5], m - 1: w[-0.5], m: w[0.5], m + 1: w[1.5]}
        for pos, wt in taps.items():
            D[m] += wt * E[pos + 3]
    return D


def _kron_axis(mats, ax, shape):
    """Operator acting along axis `ax` of a (x, y[, z]) grid flattened x-fastest."""
    out = np.ones((1, 1))
    for a in reversed(range(len(shape))):
        out = np.kron(out, mats if a == ax else np.eye(shape[a]))
    return out


def _oracle_maps(shape, bc):
    """Extract G_c (p -> v_c) and D_c (v_c -> p) from oracle impulse runs in FP64
    with unit coefficients: one step with b = 0 gives v = G p; with a = 0 it
    gives p = D v."""
    nd = len(shape)
    npts = int(np.prod(shape))
    cfg = O.acoustic_cfg(shape, bc, O.FP64, 0)
    G = [np.zeros((npts, npts)) for _ in range(nd)]
    D = [np.zeros((npts, npts)) for _ in range(nd)]
    for q in range(npts):
        st = O.AcousticState(cfg)
        st.p.flat[q] = 1.0
        st.a = [np.ones(st.shape) for _ in range(3)]
        st.b = np.zeros(st.shape)
        st.run(1)
        for c in range(nd):
            G[c][:, q] = st.v[c].ravel()
        for c in range(nd):
            st = O.AcousticState(cfg)
            st.v[c].flat[q] = 1.0
            st.a = [np.zeros(st.shape) for _ in range(3)]
            st.b = np.ones(st.shape)
            st.run(1)
            D[c][:, q] = st.p.ravel()
    return G, D


CASES = [((8, 8), (O.BC_RIGID, O.BC_RIGID)),
         ((8, 8), (O.BC_PERIODIC, O.BC_PERIODIC)),
         ((8, 7), (O.BC_PERIODIC, O.BC_RIGID)),
         ((5, 6, 4), (O.BC_RIGID, O.BC_PERIODIC, O.BC_RIGID))]


@pytest.mark.parametrize("shape,bc", CASES)
def test_operators_match_stencil_and_are_skew(oracle_lib, shape, bc):
    G, D = _oracle_maps(shape, bc)
    for c in range(len(shape)):
        G_ref = _kron_axis(_diff_1d(shape[c], bc[c], True), c, shape)
        D_ref = _kron_axis(_diff_1d(shape[c], bc[c], False), c, shape)
        # the oracle masks wall values of the velocity in the other axes only
        # through its initial data; the operator itself is the plain stencil
        np.testing.assert_array_equal(G[c], G_ref)
        np.testing.assert_array_equal(D[c], D_ref)
        # skew structure on the unknowns that are not held at zero by rigid
        # walls: gradient = - divergence^T, exactly
        pm, vm = _active(shape, bc, c)
        np.testing.assert_array_equal(G[c][np.ix_(vm, pm)], -D[c][np.ix_(pm, vm)].T)
        # and the held-at-zero p wall nodes receive nothing from the free v_c
        assert not np.any(D[c][np.ix_(~pm, vm)])


def _active(shape, bc, c):
    """Masks of p nodes and v_c points that are free unknowns: p is zero on
    every rigid wall node plane (index 0), v_c on the wall planes of the rigid
    axes other than c."""
    idx = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    idx = [i.transpose().ravel() for i in idx]      # flattened x-fastest
    pm = np.ones(idx[0].size, bool)
    vm = np.ones(idx[0].size, bool)
    for ax, b in enumerate(bc):
        if b == O.BC_RIGID:
            pm &= idx[ax] != 0
            if ax != c:
                vm &= idx[ax] != 0
    return pm, vm


def test_interior_impulse_response_is_the_printed_stencil(oracle_lib):
    """The divergence of a single v impulse at an interior point reproduces
    the printed weights [1/24, -9/8, 9/8, -1/24] at the four p nodes."""
    shape = (12, 12)
    cfg = O.acoustic_cfg(shape, (O.BC_PERIODIC, O.BC_PERIODIC), O.FP64, 0)
    st = O.AcousticState(cfg)
    st.a = [np.zeros(st.shape) for _ in range(3)]
    st.b = np.ones(st.shape)
    st.v[0][5, 5] = 1.0     # vx at x = 5 + 1/2, y = 5
    st.run(1)
    row = st.p[5]
    # node m reads vx[m-2], vx[m-1], vx[m], vx[m+1] at offsets -3/2, -1/2,
    # +1/2, +3/2, so the impulse at vx[5] (x = 5 + 1/2) reaches nodes 4..7
    w = _weights()
    expect = np.zeros(12)
    expect[4] = w[1.5]
    expect[5] = w[0.5]
    expect[6] = w[-0.5]
    expect[7] = w[-1.5]
    np.testing.assert_array_equal(row, expect)
    assert np.count_nonzero(st.p) == 4


def _amplification(shape, bc, cfl):
    """One leapfrog step as a dense matrix on (p, v_1..v_d), built from oracle
    impulse runs with a = b = cfl (FP64)."""
    nd = len(shape)
    npts = int(np.prod(shape))
    cfg = O.acoustic_cfg(shape, bc, O.FP64, 0)
    nstate = npts * (nd + 1)
    M = np.zeros((nstate, nstate))
    for col in range(nstate):
        st = O.AcousticState(cfg)
        st.a = [np.full(st.shape, cfl) for _ in range(3)]
        st.b = np.full(st.shape, cfl)
        f, q = divmod(col, npts)
        (st.p if f == 0 else st.v[f - 1]).flat[q] = 1.0
        st.run(1)
        M[:, col] = np.concatenate([st.p.ravel()] + [st.v[c].ravel() for c in range(nd)])
    return M


@pytest.mark.parametrize("shape,bc", [((8, 8), (O.BC_PERIODIC, O.BC_PERIODIC)),
                                      ((8, 8), (O.BC_RIGID, O.BC_RIGID))])
def test_amplification_on_unit_circle_below_cfl_limit(oracle_lib, shape, bc):
    # 2D limit of the 4th-order staggered scheme: 1 / (sqrt(2) (9/8 + 1/24)) = 0.606
    lam = np.linalg.eigvals(_amplification(shape, bc, 0.5))
    assert np.max(np.abs(lam)) < 1.0 + 1e-6
    assert np.min(np.abs(lam)) > 1.0 - 1e-6
    lam_unstable = np.linalg.eigvals(_amplification(shape, bc, 0.7))
    assert np.max(np.abs(lam_unstable)) > 1.01
