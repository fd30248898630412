"""The allocation-free rescale entry point (for callers that cannot allocate
device memory, e.g. while a stream is captured or under a fixed memory
budget) must give exactly the ciphertexts of the ordinary rescale, on two
calls in a row that reuse its fixed scratch array, and must refuse sizes
beyond that array. Collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2409_07751_gb300 import build, ckks
    build.build()
    return ckks


def test_rescale_noalloc_matches_rescale_twice(G):
    import torch
    ctx = G.Context(13, 6, 2)
    keys = G.Keys(ctx, 5)
    rng = np.random.default_rng(4)
    for call, (level, batch) in enumerate([(6, 2), (3, 3)]):
        v = rng.uniform(-1, 1, (batch, 100))
        ct = G.encrypt(ctx, keys, v, level, seed=10 + call)
        ref = G.rescale(ctx, ct).export()
        din = torch.from_numpy(ct.export().view(np.int64).copy()).cuda()
        dout = torch.full(ref.shape, -1, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        G.rescale_noalloc(ctx, din.data_ptr(), batch, level, dout.data_ptr())
        ctx.synchronize()
        got = dout.cpu().numpy().view(np.uint64)
        assert (got == ref).all(), call


def test_rescale_noalloc_rejects_oversize(G):
    import torch
    ctx = G.Context(16, 2, 1)
    d = torch.zeros(16, dtype=torch.int64, device="cuda")
    # 2 * 64 * 65536 * (1 + 1) words > 8 Mi words
    with pytest.raises(G.CkksError) as e:
        G.rescale_noalloc(ctx, d.data_ptr(), 64, 1, d.data_ptr())
    assert e.value.code == -1
