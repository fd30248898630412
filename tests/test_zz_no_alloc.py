"""The allocation-free rescale entry point (for callers that cannot allocate
device memory, e.g. while a stream is captured or under a fixed memory
budget) must give exactly the ciphertexts of the ordinary rescale, on two
calls in a row that reuse its fixed scratch array, must take no memory from
the device's stream-ordered pool (the one the library allocates from), and
must refuse sizes beyond that array, sizes whose word count would wrap
around, and overlapping input and output. Collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# CUmemPool_attribute values of the driver API (cuda.h)
_USED_MEM_CURRENT, _USED_MEM_HIGH = 7, 8


@pytest.fixture(scope="module")
def G():
    from paper_2409_07751_gb300 import build, ckks
    build.build()
    return ckks


class _Pool:
    """The current device's default memory pool through the driver API."""

    def __init__(self):
        import torch
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        z = ctypes.c_uint64(0)  # resets the high watermark to the current use
        assert self.cu.cuMemPoolSetAttribute(self.pool, _USED_MEM_HIGH, ctypes.byref(z)) == 0


def test_rescale_noalloc_matches_rescale_twice(G):
    import torch
    ctx = G.Context(13, 6, 2)
    keys = G.Keys(ctx, 5)
    rng = np.random.default_rng(4)
    pool = _Pool()
    for call, (level, batch) in enumerate([(6, 2), (3, 3)]):
        v = rng.uniform(-1, 1, (batch, 100))
        ct = G.encrypt(ctx, keys, v, level, seed=10 + call)
        ref = G.rescale(ctx, ct).export()
        din = torch.from_numpy(ct.export().view(np.int64).copy()).cuda()
        dout = torch.full(ref.shape, -1, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        ctx.synchronize()
        before = pool.get(_USED_MEM_CURRENT)
        pool.reset_high()
        G.rescale_noalloc(ctx, din.data_ptr(), batch, level, dout.data_ptr())
        ctx.synchronize()
        # nothing taken from the pool, not even briefly inside the call
        assert pool.get(_USED_MEM_HIGH) == before, call
        assert pool.get(_USED_MEM_CURRENT) == before, call
        got = dout.cpu().numpy().view(np.uint64)
        assert (got == ref).all(), call


def test_rescale_noalloc_rejects_bad_sizes_and_overlap(G):
    import torch
    ctx = G.Context(16, 2, 1)
    d = torch.zeros(16, dtype=torch.int64, device="cuda")
    dev = torch.cuda.current_device()
    # 2 * 64 * 65536 * (1 + 1) words > 8 Mi words
    for batch in (64, 2 ** 47 + 1, 2 ** 62):  # the last two wrap a size_t product
        with pytest.raises(G.CkksError) as e:
            G.rescale_noalloc(ctx, d.data_ptr(), batch, 1, d.data_ptr())
        assert e.value.code == -1, batch
    # in place: the output limbs would overwrite input limbs still to be read
    small = G.Context(10, 3, 1)
    buf = torch.zeros(2 * 4 * 1024, dtype=torch.int64, device="cuda")
    with pytest.raises(G.CkksError) as e:
        G.rescale_noalloc(small, buf.data_ptr(), 1, 3, buf.data_ptr())
    assert e.value.code == -1
    assert torch.cuda.current_device() == dev
