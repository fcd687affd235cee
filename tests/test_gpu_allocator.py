"""The caller-allocator hook (wave_set_allocator) on the GPU: device memory
from torch's caching allocator gives the same bits as the library's own
allocations and is all returned on destroy; a hook that returns NULL (a
failure injected on the host, no GPU fault) makes wave_create fail with
ENOMEM after freeing everything it had allocated, and the device stays usable."""
import numpy as np
import pytest

from paper_2310_00236_gb300 import inputs
from paper_2310_00236_gb300 import wave as W
from wave_helpers import gpu_bits

pytestmark = pytest.mark.gpu

SHAPE = (64, 32, 40)


class Hook:
    """Counting allocator over torch's caching allocator; allocation number
    fail_at (1-based) returns NULL."""

    def __init__(self, fail_at=0):
        import torch
        self.torch = torch
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}
        self.cbs = (W.ALLOC_FN(self.alloc), W.FREE_FN(self.free))

    def alloc(self, nbytes, stream, user):
        self.calls += 1
        if self.calls == self.fail_at:
            return None
        p = self.torch.cuda.caching_allocator_alloc(int(nbytes), 0, stream or 0)
        self.live[p] = int(nbytes)
        return p

    def free(self, ptr, nbytes, stream, user):
        assert self.live.pop(ptr) == nbytes
        self.torch.cuda.caching_allocator_delete(ptr)

    def install(self):
        W._check(W.lib().wave_set_allocator(self.cbs[0], self.cbs[1], None))


def _create():
    h = 10.0
    c = inputs.smooth_random_field(SHAPE, 4, 2.0, 1500.0, 4500.0)
    rho = np.full(c.shape, 1000.0)
    return W.wave_create(SHAPE, h, rho, c, 0.4 * h / 4500.0, W.WAVE_FP16, W.WAVE_COMP_3OP,
                         bc=[W.WAVE_BC_RIGID] * 6)


def _run():
    ctx = _create()
    try:
        W.wave_set_initial(ctx, W.WAVE_F_P, inputs.gaussian(SHAPE, 10.0, 60.0))
        W.wave_step(ctx, 9)
        return [gpu_bits(W.wave_get_raw(ctx, f, t)) for f in range(4) for t in (0, 1)], W.wave_energy(ctx)
    finally:
        W.wave_destroy(ctx)


def test_torch_allocator_same_bits_and_all_returned():
    W.use_default_allocator()
    ref, e_ref = _run()
    hook = Hook()
    hook.install()
    try:
        got, e = _run()
    finally:
        W.use_default_allocator()
    assert hook.calls > 10 and not hook.live      # every allocation came back
    assert e == e_ref
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


def test_allocator_null_gives_enomem_and_frees_everything():
    import torch
    hook = Hook()
    hook.install()
    try:
        W.wave_destroy(_create())
    finally:
        W.use_default_allocator()
    total = hook.calls
    for k in range(1, total + 1):
        hook = Hook(fail_at=k)
        hook.install()
        try:
            with pytest.raises(W.WaveError) as e:
                _create()
        finally:
            W.use_default_allocator()
        assert e.value.status == W.WAVE_ENOMEM, (k, str(e.value))
        assert hook.calls == k and not hook.live, (k, hook.calls, len(hook.live))
    torch.cuda.synchronize()
    ref, _ = _run()                                   # the device is still usable
    assert np.any(ref[0] != 0)
