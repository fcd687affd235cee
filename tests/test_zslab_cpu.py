"""Domain decomposition along z on the host (gloo, world size 2; not in the
paper). A 3D acoustic problem (variable density and speed, p = 0 walls, a
point source, fp16 + sum_3op) is split into two slabs, one per rank; each
rank steps its slab with the oracle's half steps and exchanges two ghost
planes per cut face and half step through paper_2310_00236_gb300.zslab, the
same protocol the GPU slabs use. The slabs reproduce the whole grid's oracle
run bit for bit. (Unmeasured on hardware: every GPU call here has one GPU.)"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPE = (24, 20, 30)   # x, y, z
STEPS = 12


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem():
    import oracle as O
    from paper_2310_00236_gb300 import inputs
    nx, ny, nz = SHAPE
    h = 10.0
    c = inputs.smooth_random_field((nx, ny, nz), 7, 2.0, 1500.0, 4500.0)
    rho = inputs.smooth_random_field((nx, ny, nz), 8, 2.0, 1000.0, 2600.0)
    dt = 0.4 * h / 4500.0
    rng = np.random.default_rng(5)
    p0 = inputs.gaussian((nx, ny, nz), h, 30.0) + 0.05 * rng.standard_normal(c.shape)
    st = O.acoustic_setup(SHAPE, (1, 1, 1), h, dt, rho, c, O.FP16, 3, p0=p0)
    # physical amplitude whose scaled increment b s^ stays near 0.1 (s^ = w Z0 / h^2)
    wav = np.sin(np.arange(STEPS) * 0.7) * 0.25 * h * h / st.Z0
    st.src_index = 11 + nx * (9 + ny * 16)          # node (11, 9, 16): in the upper slab
    st.src = O.scale_source(wav, st.Z0, 1.0, h, 3, O.FP16)
    return st


class OracleSlab:
    """The oracle's slab of planes [z0, z1) of the whole state, as a zslab stepper."""

    def __init__(self, whole, z0, z1):
        import oracle as O
        import torch
        nz = SHAPE[2]
        cfg = O.acoustic_cfg(SHAPE[:2] + (z1 - z0,), (1, 1, 1), O.FP16, 3)
        st = O.AcousticState(cfg)
        cut = lambda a: np.ascontiguousarray(a[z0:z1])
        st.p, st.tp = cut(whole.p), cut(whole.tp)
        st.v = [cut(x) for x in whole.v]
        st.tv = [cut(x) for x in whole.tv]
        st.a = [cut(x) for x in whole.a]
        st.b = cut(whole.b)
        src_k = whole.src_index // (SHAPE[0] * SHAPE[1])
        st.src_index = whole.src_index - z0 * SHAPE[0] * SHAPE[1] if z0 <= src_k < z1 else -1
        st.src = whole.src
        self.st, self.O = st, O
        shape = (2, SHAPE[1], SHAPE[0])
        self.g = {f: (torch.zeros(shape, dtype=torch.float64) if z0 > 0 else None,
                      torch.zeros(shape, dtype=torch.float64) if z1 < nz else None) for f in ("p", "vz")}

    def _arr(self, field):
        return self.st.p if field == "p" else self.st.v[2]

    def edges(self, field):
        import torch
        a = self._arr(field)
        return torch.from_numpy(a[:2].copy()), torch.from_numpy(a[-2:].copy())

    def ghosts(self, field):
        return self.g[field]

    def half_step(self, which):
        lo, hi = self.g["p" if which == 0 else "vz"]
        self.O.acoustic_half_step(self.st, which, None if lo is None else lo.numpy(),
                                  None if hi is None else hi.numpy())


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from paper_2310_00236_gb300 import zslab
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        whole = _problem()
        z0, z1 = zslab.slab_bounds(SHAPE[2], ws, rank)
        slab = OracleSlab(whole, z0, z1)
        zslab.run(slab, STEPS, lambda s, f: zslab.exchange(s, f, rank, ws))
        s = slab.st
        out.put((rank, z0, z1, s.p, s.tp, [x.copy() for x in s.v], [x.copy() for x in s.tv]))
    finally:
        dist.destroy_process_group()


def test_two_slabs_over_gloo_reproduce_the_whole_grid(oracle_lib):
    import torch.multiprocessing as mp
    ref = _problem()
    ref.run(STEPS)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    assert np.all(np.isfinite(ref.p)) and np.all(np.isfinite(ref.tv[2]))
    covered = 0
    for rank, z0, z1, p, tp, v, tv in sorted(got, key=lambda g: g[0]):
        np.testing.assert_array_equal(p, ref.p[z0:z1])
        np.testing.assert_array_equal(tp, ref.tp[z0:z1])
        for c in range(3):
            np.testing.assert_array_equal(v[c], ref.v[c][z0:z1])
            np.testing.assert_array_equal(tv[c], ref.tv[c][z0:z1])
        covered += z1 - z0
    assert covered == SHAPE[2]
    # the source (upper slab) has reached the lower slab through the exchanges
    assert np.any(ref.p[14] != _problem().p[14])


def test_slab_bounds():
    from paper_2310_00236_gb300 import zslab
    assert [zslab.slab_bounds(30, 2, r) for r in range(2)] == [(0, 15), (15, 30)]
    assert [zslab.slab_bounds(35, 4, r) for r in range(4)] == [(0, 9), (9, 18), (18, 27), (27, 35)]
    with pytest.raises(ValueError):
        zslab.slab_bounds(30, 4, 0)


def test_slab_without_exchange_differs(oracle_lib):
    """Planted mistake: the same two slabs with ghost planes left at zero (no
    exchange) do not reproduce the whole grid."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from paper_2310_00236_gb300 import zslab
    ref = _problem()
    ref.run(STEPS)
    whole = _problem()
    slabs = [OracleSlab(whole, *zslab.slab_bounds(SHAPE[2], 2, r)) for r in range(2)]
    zslab.run(slabs[0], STEPS, lambda s, f: None)
    assert np.any(slabs[0].st.p != ref.p[:15])
    # and with the in-process exchange they do
    whole = _problem()
    slabs = [OracleSlab(whole, *zslab.slab_bounds(SHAPE[2], 2, r)) for r in range(2)]
    zslab.exchange_local(slabs, "p")
    for _ in range(STEPS):
        for s in slabs:
            s.half_step(0)
        zslab.exchange_local(slabs, "vz")
        for s in slabs:
            s.half_step(1)
        zslab.exchange_local(slabs, "p")
    np.testing.assert_array_equal(np.concatenate([s.st.p for s in slabs]), ref.p)
    np.testing.assert_array_equal(np.concatenate([s.st.tv[2] for s in slabs]), ref.tv[2])
