"""Domain decomposition of a 3D acoustic grid along z (not in the paper).

A grid of nz planes is cut into slabs of consecutive planes, one per GPU (one
process per GPU). Section 3's fourth-order staggered stencil reaches two points
past a node, so every half step needs two ghost planes per cut face of the field
it differentiates along z: p before the velocity half step, v_z before the
pressure half step. A step is therefore

    half_step(0); exchange("vz"); half_step(1); exchange("p")

with one exchange of p before the first step. Compensations are point-local and
are never exchanged. Each slab sends its first two planes down (the lower
neighbour's upper ghosts) and its last two planes up (the upper neighbour's
lower ghosts), into the receiver's own buffers; no process reads another GPU's
memory.

This module holds the host side: the slab bounds, the exchange over
torch.distributed (NCCL between GPUs, gloo on the host), the step sequence, and
`Slab`, a stepper over one slab context of the C ABI (wave_create with
z_cut / z0 / rho_above, wave_set_z_ghosts, wave_half_step, wave_copy_planes).
A stepper is any object with half_step(which), edges(field) -> (first two
planes, last two planes) and ghosts(field) -> (lower ghost buffer, upper ghost
buffer), where field is "p" or "vz".
"""
from __future__ import annotations

import numpy as np

from . import wave as W

FIELDS = {"p": W.WAVE_F_P, "vz": W.WAVE_F_VZ}


def slab_bounds(nz: int, world: int, rank: int, min_planes: int = 8):
    """Planes [z0, z1) of slab `rank` when nz planes are split as evenly as
    possible over `world` slabs (the first nz % world slabs get one more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world / rank")
    base, extra = divmod(nz, world)
    if base < min_planes:
        raise ValueError(f"{nz} planes over {world} slabs leaves fewer than {min_planes} per slab")
    z0 = rank * base + min(rank, extra)
    return z0, z0 + base + (1 if rank < extra else 0)


def exchange(stepper, field: str, rank: int, world: int, group=None):
    """Send this slab's edge planes of `field` to its neighbours and receive
    theirs into the ghost buffers (torch.distributed point-to-point)."""
    import torch.distributed as dist
    lo2, hi2 = stepper.edges(field)
    glo, ghi = stepper.ghosts(field)
    ops = []
    if rank > 0:
        ops += [dist.P2POp(dist.isend, lo2, rank - 1, group), dist.P2POp(dist.irecv, glo, rank - 1, group)]
    if rank < world - 1:
        ops += [dist.P2POp(dist.isend, hi2, rank + 1, group), dist.P2POp(dist.irecv, ghi, rank + 1, group)]
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


def exchange_local(steppers, field: str):
    """The same exchange between slabs held by one process (in order of z),
    by copies: slab i's last two planes become slab i+1's lower ghosts and slab
    i+1's first two planes slab i's upper ghosts."""
    edges = [s.edges(field) for s in steppers]
    for i in range(len(steppers) - 1):
        steppers[i + 1].ghosts(field)[0].copy_(edges[i][1])
        steppers[i].ghosts(field)[1].copy_(edges[i + 1][0])


def run(stepper, nsteps: int, comm, first: bool = True):
    """nsteps leapfrog steps of one slab; comm(stepper, field) exchanges.
    first: exchange p before the first step (the ghosts start empty)."""
    if first:
        comm(stepper, "p")
    for _ in range(nsteps):
        stepper.half_step(0)
        comm(stepper, "vz")
        stepper.half_step(1)
        comm(stepper, "p")


class Slab:
    """One z slab of a 3D acoustic grid on the current GPU.

    n_global: cells per axis (x, y, z) of the whole grid; z0, z1: this slab's
    planes. rho, c: the whole grid's materials (shape (nz, ny, nx)), of which the
    slab takes its planes and, when its upper face is a cut, the plane above it;
    Z0 = max(rho) * max(c) of the whole grid, so every slab uses the same units.
    bc: the grid's face codes (the z faces apply only where the slab reaches
    them). The context steps with the streaming kernels (the slab needs n[0] a
    multiple of the 16-byte vector width).
    """

    def __init__(self, n_global, z0: int, z1: int, h: float, rho, c, dt: float, precision: int, comp: int,
                 bc=(W.WAVE_BC_RIGID,) * 6, field_scale: float = 1.0, stream=None):
        import torch
        nx, ny, nz = n_global
        self.z0, self.z1 = z0, z1
        self.cut = (1 if z0 > 0 else 0) | (2 if z1 < nz else 0)
        rho = np.asarray(rho, dtype=np.float64)
        c = np.asarray(c, dtype=np.float64)
        z0_scale = float(rho.max() * c.max())
        above = rho[z1] if z1 < nz else None
        self.ctx = W.wave_create((nx, ny, z1 - z0), h, rho[z0:z1], c[z0:z1], dt, precision, comp, bc=bc,
                                 field_scale=field_scale, kernel=2, stream=stream, z_cut=self.cut,
                                 z0=z0_scale, rho_above=above)
        pitch, plane, eb = W.wave_get_layout(self.ctx)
        dtype = torch.float32 if eb == 4 else torch.int16
        buf = lambda: torch.zeros((2, plane), dtype=dtype, device="cuda")
        self._ghost = {f: (buf() if self.cut & 1 else None, buf() if self.cut & 2 else None) for f in FIELDS}
        self._edge = {f: (buf(), buf()) for f in FIELDS}
        W.wave_set_z_ghosts(self.ctx, self._ghost["p"][0], self._ghost["p"][1], self._ghost["vz"][0],
                            self._ghost["vz"][1])

    def half_step(self, which: int):
        W.wave_half_step(self.ctx, which)

    def edges(self, field: str):
        lo, hi = self._edge[field]
        nzl = self.z1 - self.z0
        W.wave_copy_planes(self.ctx, FIELDS[field], 0, 2, lo)
        W.wave_copy_planes(self.ctx, FIELDS[field], nzl - 2, 2, hi)
        return lo, hi

    def ghosts(self, field: str):
        return self._ghost[field]

    def destroy(self):
        W.wave_destroy(self.ctx)
