"""torch.autograd.Function over the C ABI: pressure traces of an acoustic run
as a function of the velocity model, with the gradient from the discrete
adjoint (wave_record / wave_adjoint_step / wave_get_gradient).

Not in the paper. Every step runs in the library's CUDA kernels; this module
only marshals arguments and owns the context between forward and backward.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import wave as W


@dataclass
class Shot:
    """One acoustic experiment. shape: cells (x, y[, z]); rho: density shaped
    like a field ((z,) y, x); src_idx: source node (i, j[, k]) with wavelet
    (physical units, one sample per step); rec_idx: receiver nodes; nsteps:
    steps recorded; ncheckpoints: 0 for ceil(sqrt(nsteps))."""
    shape: tuple
    h: float
    dt: float
    rho: np.ndarray
    src_idx: tuple
    wavelet: np.ndarray
    rec_idx: list
    nsteps: int
    precision: int = W.WAVE_FP16
    comp: int = W.WAVE_COMP_3OP
    bc: tuple = (W.WAVE_BC_RIGID,) * 6
    field_scale: float = 1.0
    ncheckpoints: int = 0
    stream: object = None
    p0: np.ndarray | None = field(default=None)


class _Holder:
    """Destroys the context when the autograd graph releases it."""

    def __init__(self, ctx):
        self.ctx = ctx

    def close(self):
        if self.ctx is not None:
            W.wave_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        self.close()


def record(c: np.ndarray, shot: Shot):
    """Create the context for velocity model c, run the recorded forward
    pass. Returns (holder, traces [nsteps, nrec] float32 CUDA tensor)."""
    ctx = W.wave_create(shot.shape, shot.h, shot.rho, c, shot.dt, shot.precision, shot.comp,
                        bc=list(shot.bc), field_scale=shot.field_scale, stream=shot.stream)
    holder = _Holder(ctx)
    if shot.p0 is not None:
        W.wave_set_initial(ctx, W.WAVE_F_P, shot.p0)
    if shot.wavelet is not None and len(shot.wavelet):
        W.wave_set_source(ctx, W.WAVE_F_P, shot.src_idx, shot.wavelet)
    nrec = len(shot.rec_idx)
    traces = torch.zeros((shot.nsteps, nrec), dtype=torch.float32, device="cuda")
    if nrec:
        W.wave_set_receivers(ctx, W.WAVE_F_P, shot.rec_idx, traces, shot.nsteps)
    W.wave_record(ctx, shot.nsteps, shot.ncheckpoints)
    return holder, traces


class AcousticTraces(torch.autograd.Function):
    """traces = F(c) for one Shot; dJ/dc = F'(c)^T dJ/dtraces by the adjoint."""

    @staticmethod
    def forward(fctx, c: torch.Tensor, shot: Shot):
        c_np = c.detach().to(torch.float64).cpu().numpy()
        holder, traces = record(c_np, shot)
        fctx.holder = holder
        fctx.c_meta = (c.dtype, c.device, c.shape)
        fctx.nsteps = shot.nsteps
        return traces

    @staticmethod
    def backward(fctx, grad_traces: torch.Tensor):
        holder = fctx.holder
        if holder.ctx is None:
            raise RuntimeError("AcousticTraces.backward called twice (the adjoint consumes the run)")
        res = grad_traces.detach().to(device="cuda", dtype=torch.float32).contiguous()
        W.wave_adjoint_step(holder.ctx, fctx.nsteps, res)
        g, left = W.wave_get_gradient(holder.ctx)
        torch.cuda.current_stream().synchronize()
        holder.close()
        dtype, device, shape = fctx.c_meta
        return g.reshape(shape).to(device=device, dtype=dtype), None


def traces(c: torch.Tensor, shot: Shot) -> torch.Tensor:
    """Differentiable pressure traces [nsteps, nrec] of `shot` for velocity c."""
    return AcousticTraces.apply(c, shot)
