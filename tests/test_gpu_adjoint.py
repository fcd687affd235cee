"""GPU discrete adjoint (gradient of a trace misfit with respect to the
velocity model) against the binary64 oracle adjoint, which is itself pinned by
the dot-product identity and central differences (test_oracle_adjoint.py).

* binary32 forward + adjoint: dJ/dc within 1e-4 (relative L2) of the oracle;
* binary16 + sum_3op forward (binary32 adjoint): within the accuracy of the
  half-precision forward run (the recorded traces themselves are bit-exact
  with the oracle's emulation of the same run);
* checkpoint counts and splits of the adjoint into several calls give the
  same bits (the replayed forward segments are bit-identical);
* the torch.autograd.Function gives the same bits as the C ABI sequence, and
  central differences of the GPU misfit agree with the GPU gradient.
"""
import numpy as np
import pytest

import oracle as O
from paper_2310_00236_gb300 import inputs
from paper_2310_00236_gb300 import wave as W
from wave_helpers import PREC, to_bits

pytestmark = pytest.mark.gpu
R, P = W.WAVE_BC_RIGID, W.WAVE_BC_PERIODIC


def _case(shape, bc, nsteps, seed=0, const_rho=False):
    """Smooth random true and start models, Ricker source near the y = 0 (2D)
    or z = 0 (3D) face, receivers at seeded nodes (one on a wall node, two
    sharing a point)."""
    nd = len(shape)
    h = 10.0
    dt = 0.4 * h / 4500.0
    if const_rho:
        rho = np.full(tuple(shape[::-1]), 1000.0)
    else:
        rho = 1000.0 + 200.0 * inputs.smooth_random_field(shape, seed + 7, 2.0, -1.0, 1.0)
    c_true = inputs.smooth_random_field(shape, seed + 1, 3.0, 1500.0, 4500.0)
    c0 = 0.7 * c_true + 0.3 * inputs.smooth_random_field(shape, seed + 2, 6.0, 1500.0, 4500.0)
    z0 = float(rho.max() * 4500.0)
    hd1 = h if nd == 2 else h * h
    wav = 0.5 * hd1 / z0 * inputs.ricker_table(nsteps, dt, 1.0 / (25 * dt))
    src = tuple(s // 2 for s in shape[:-1]) + (2,)
    rng = np.random.default_rng(seed + 3)
    rec = [tuple(int(rng.integers(1, s - 1)) for s in shape) for _ in range(9)]
    rec.append(tuple([0] + [s // 3 for s in shape[1:]]))  # on the x = 0 face
    rec.append(rec[1])  # two receivers on one point
    return dict(shape=shape, bc=bc, nd=nd, h=h, dt=dt, rho=rho, c_true=c_true, c0=c0, wav=wav,
                src=src, rec=rec, nsteps=nsteps)


def _lin(shape, idx):
    return int(np.ravel_multi_index(tuple(idx[::-1]), tuple(shape[::-1])))


def _oracle_state(k, c, fmt=O.FP64, comp=0):
    st = O.acoustic_setup(k["shape"], k["bc"], k["h"], k["dt"], k["rho"], c, fmt, comp, P0=1.0)
    st.src_index = _lin(k["shape"], k["src"])
    st.src = O.scale_source(k["wav"], st.Z0, 1.0, k["h"], k["nd"], fmt)
    return st


def _observed(k):
    st = _oracle_state(k, k["c_true"])
    tr, _ = st.run(k["nsteps"], 0, [_lin(k["shape"], r) for r in k["rec"]])
    return tr


def _gpu_gradient(k, prec, comp, d_obs, ncp=0, splits=None, kernel=0):
    import torch
    code = PREC[prec][0]
    ctx = W.wave_create(k["shape"], k["h"], k["rho"], k["c0"], k["dt"], code, comp,
                        bc=[b for b in k["bc"] for _ in range(2)] + [0] * (6 - 2 * k["nd"]), kernel=kernel)
    try:
        W.wave_set_source(ctx, W.WAVE_F_P, k["src"], k["wav"])
        n, nrec = k["nsteps"], len(k["rec"])
        tr = torch.zeros((n, nrec), dtype=torch.float32, device="cuda")
        W.wave_set_receivers(ctx, W.WAVE_F_P, k["rec"], tr, n)
        W.wave_record(ctx, n, ncp)
        res = (tr - torch.from_numpy(d_obs).to(device="cuda", dtype=torch.float32)).contiguous()
        for m in (splits or [n]):
            W.wave_adjoint_step(ctx, m, res)
        g, left = W.wave_get_gradient(ctx)
        assert left == 0
        torch.cuda.synchronize()
        return g.cpu().numpy().astype(np.float64), tr.cpu().numpy().astype(np.float64)
    finally:
        W.wave_destroy(ctx)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [((48, 40), (R, R), 150), ((40, 32), (P, R), 120), ((24, 20, 16), (R, R, R), 60),
         ((64, 24, 16), (R, R, P), 50),
         # n[0] not a multiple of 8: the gradient kernel's last x vector is partial
         ((45, 30), (P, R), 90), ((37, 20, 12), (R, P, R), 40)]


@pytest.mark.parametrize("shape,bc,nsteps", CASES)
def test_adjoint_fp32_matches_oracle(shape, bc, nsteps):
    k = _case(shape, bc, nsteps)
    d_obs = _observed(k)
    g, tr = _gpu_gradient(k, "fp32", 0, d_obs)
    ref = O.acoustic_adjoint(_oracle_state(k, k["c0"]), k["c0"], nsteps,
                             [_lin(shape, r) for r in k["rec"]], d_obs=d_obs)
    assert np.all(np.isfinite(g))
    assert _rel(tr, ref["traces"]) < 1e-5
    assert _rel(g, ref["grad_c"]) < 1e-4, _rel(g, ref["grad_c"])


@pytest.mark.parametrize("shape,bc,nsteps", [CASES[0], CASES[3]])
def test_adjoint_fp16_kahan_traces_exact_and_gradient_close(shape, bc, nsteps):
    k = _case(shape, bc, nsteps)
    d_obs = _observed(k)
    g, tr = _gpu_gradient(k, "fp16", 3, d_obs)
    # the recorded traces are the oracle's emulation of the same fp16 run, bit for bit
    emu = _oracle_state(k, k["c0"], O.FP16, 3)
    tr_emu, _ = emu.run(nsteps, 0, [_lin(shape, r) for r in k["rec"]])
    assert np.array_equal(tr, tr_emu)
    ref = O.acoustic_adjoint(_oracle_state(k, k["c0"]), k["c0"], nsteps,
                             [_lin(shape, r) for r in k["rec"]], d_obs=d_obs)
    assert _rel(g, ref["grad_c"]) < 5e-2, _rel(g, ref["grad_c"])


@pytest.mark.parametrize("prec,comp,const_rho", [("fp32", 0, False), ("fp16", 3, False), ("bf16", 6, False),
                                                 ("fp16", 3, True)])
def test_adjoint_checkpoints_and_splits_bit_identical(prec, comp, const_rho):
    # constant density and a rigid x axis with n[0] = 64 take the one-pass 3D
    # kernel (ping-pong buffers) in the forward replays
    k = _case((64, 24, 16), (R, R, P), 37, const_rho=const_rho)
    d_obs = _observed(k)
    g0, _ = _gpu_gradient(k, prec, comp, d_obs, ncp=0)
    for ncp, splits in ((1, None), (5, [7, 30]), (37, [1] * 37), (0, [36, 1])):
        g, _ = _gpu_gradient(k, prec, comp, d_obs, ncp=ncp, splits=splits)
        assert np.array_equal(g, g0), (ncp, splits)


@pytest.mark.parametrize("prec,comp", [("fp16", 3), ("fp32", 0)])
def test_one_pass_adjoint_equals_two_kernel_adjoint(prec, comp):
    """Constant density, rigid x and n[0] = 64: the adjoint sweep runs the
    one-pass step on ping-pong buffers (kernel 0); with the streaming kernels
    forced (kernel 2) it runs the two half steps. Same gradient bits."""
    k = _case((64, 24, 16), (R, R, P), 23, const_rho=True)
    d_obs = _observed(k)
    g_one, tr_one = _gpu_gradient(k, prec, comp, d_obs, ncp=4, splits=[9, 14])
    g_two, tr_two = _gpu_gradient(k, prec, comp, d_obs, ncp=4, splits=[9, 14], kernel=2)
    assert np.array_equal(tr_one, tr_two)
    assert np.array_equal(g_one, g_two)
    assert np.abs(g_one).max() > 0


def test_autograd_function_matches_abi_and_oracle():
    import torch
    from paper_2310_00236_gb300 import autograd as AG
    k = _case((48, 40), (R, R), 120)
    d_obs = _observed(k)
    shot = AG.Shot(shape=k["shape"], h=k["h"], dt=k["dt"], rho=k["rho"], src_idx=k["src"],
                   wavelet=k["wav"], rec_idx=k["rec"], nsteps=k["nsteps"], precision=W.WAVE_FP32,
                   comp=0, bc=(R, R, R, R, P, P))
    c = torch.tensor(k["c0"], dtype=torch.float64, requires_grad=True)
    tr = AG.traces(c, shot)
    # binary32 misfit: its gradient (tr - d_obs) is the residual the ABI sequence uses
    J = 0.5 * ((tr - torch.from_numpy(d_obs).to(device="cuda", dtype=torch.float32)) ** 2).sum()
    J.backward()
    g_abi, _ = _gpu_gradient(k, "fp32", 0, d_obs)
    assert np.array_equal(c.grad.numpy(), g_abi)
    ref = O.acoustic_adjoint(_oracle_state(k, k["c0"]), k["c0"], k["nsteps"],
                             [_lin(k["shape"], r) for r in k["rec"]], d_obs=d_obs)
    assert _rel(c.grad.numpy(), ref["grad_c"]) < 1e-4


def test_gpu_gradient_matches_central_differences_fp32():
    import torch
    from paper_2310_00236_gb300 import autograd as AG
    k = _case((40, 36), (R, R), 100, seed=4)
    d_obs = torch.from_numpy(_observed(k)).cuda()

    def J(c):
        shot = AG.Shot(shape=k["shape"], h=k["h"], dt=k["dt"], rho=k["rho"], src_idx=k["src"],
                       wavelet=k["wav"], rec_idx=k["rec"], nsteps=k["nsteps"],
                       precision=W.WAVE_FP32, comp=0, bc=(R, R, R, R, P, P))
        ct = torch.tensor(c, dtype=torch.float64, requires_grad=True)
        val = 0.5 * ((AG.traces(ct, shot).double() - d_obs) ** 2).sum()
        val.backward()
        return float(val.detach()), ct.grad.numpy()

    J0, g = J(k["c0"])
    for seed in (31, 32):
        dc = inputs.smooth_random_field(k["shape"], seed, 3.0, -1.0, 1.0)
        eps = 20.0  # m/s: large enough that the binary32 misfit noise stays well below the change
        fd = (J(k["c0"] + eps * dc)[0] - J(k["c0"] - eps * dc)[0]) / (2 * eps)
        an = float(np.sum(g * dc))
        assert abs(fd - an) <= 2e-2 * abs(an), (fd, an)


def test_adjoint_state_errors():
    import torch
    k = _case((32, 24), (R, R), 10)
    ctx = W.wave_create(k["shape"], k["h"], k["rho"], k["c0"], k["dt"], W.WAVE_FP32, 0,
                        bc=[R, R, R, R, P, P])
    try:
        with pytest.raises(W.WaveError) as ei:
            W.wave_adjoint_step(ctx, 1, None)
        assert ei.value.status == W.WAVE_ESTATE
        W.wave_record(ctx, 10, 0)
        with pytest.raises(W.WaveError) as ei:
            W.wave_adjoint_step(ctx, 11, None)
        assert ei.value.status == W.WAVE_EINVAL
        W.wave_adjoint_step(ctx, 10, None)  # no receivers: zero gradient
        g, left = W.wave_get_gradient(ctx)
        assert left == 0 and float(torch.abs(g).max()) == 0.0
    finally:
        W.wave_destroy(ctx)


def test_reset_reuses_context_across_shots_bit_exact():
    """wave_reset + a new source on one context gives the bits of a fresh
    context for each shot (forward traces and gradient), with the adjoint
    buffers of the previous shot reused."""
    import torch
    k = _case((64, 24, 16), (R, R, P), 30, const_rho=True)
    d_obs = _observed(k)
    fresh, _ = _gpu_gradient(k, "fp16", 3, d_obs)
    ctx = W.wave_create(k["shape"], k["h"], k["rho"], k["c0"], k["dt"], W.WAVE_FP16, 3,
                        bc=[b for b in k["bc"] for _ in range(2)])
    try:
        grads = []
        for shot in range(2):
            W.wave_reset(ctx)
            W.wave_set_source(ctx, W.WAVE_F_P, k["src"], k["wav"])
            n, nrec = k["nsteps"], len(k["rec"])
            tr = torch.zeros((n, nrec), dtype=torch.float32, device="cuda")
            W.wave_set_receivers(ctx, W.WAVE_F_P, k["rec"], tr, n)
            W.wave_step(ctx, 3) if shot == 1 else None  # a stray run before the reset of the next shot
            W.wave_reset(ctx)
            W.wave_record(ctx, n, 0)
            res = (tr - torch.from_numpy(d_obs).to(device="cuda", dtype=torch.float32)).contiguous()
            W.wave_adjoint_step(ctx, n, res)
            g, _ = W.wave_get_gradient(ctx)
            grads.append(g.cpu().numpy().astype(np.float64))
        for g in grads:
            assert np.array_equal(g, fresh)
    finally:
        W.wave_destroy(ctx)
