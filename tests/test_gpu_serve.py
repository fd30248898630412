"""Serving (continuous batching): requests of two models submitted at
different times while others are mid-network must produce exactly the
ciphertexts they produce when evaluated alone; admission never exceeds the
HBM budget."""
import numpy as np
import pytest

from oracle import calibrate
from paper_2409_07751_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_2409_07751_gb300 import build, ckks as G
    build.build()
    ctx = G.Context(13, 17, 2)
    ma = calibrate.calibrate(W.make_model("t", widths=[3, 5, 2], G=3, k=2), W.uniform_inputs(64, 3), 7, [1])
    mb = calibrate.calibrate(W.make_model("t", seed=5, widths=[4, 2], G=4, k=1), W.uniform_inputs(64, 4), 5, [1])
    A, B = G.Model(ctx, ma), G.Model(ctx, mb)
    ka = G.Keys(ctx, 11, A.rotations())
    kb = G.Keys(ctx, 12, B.rotations())
    return G, ctx, (A, ka, 3), (B, kb, 4)


def _req(G, ctx, keys, n_in, i, level):
    x = W.uniform_inputs(1, n_in, seed=100 + i)[0]
    return G.encrypt(ctx, keys, x, level, W.SEED_ENC, i)


def test_mix_equals_alone(env):
    G, ctx, (A, ka, na), (B, kb, nb) = env
    srv = G.Server(ctx, 1 << 40)
    ida, idb = srv.add_model(A, ka), srv.add_model(B, kb)
    plan = [  # (step at which the request arrives, model, level)
        (0, 0, 17), (0, 1, 17), (1, 0, 16), (1, 0, 17), (2, 1, 15), (3, 0, 17)]
    reqs, step = [], 0
    while step < 12:
        for i, (s, mdl, lv) in enumerate(plan):
            if s == step:
                mk, keys, n = (A, ka, na) if mdl == 0 else (B, kb, nb)
                ct = _req(G, ctx, keys, n, i, lv)
                rid = srv.submit(ida if mdl == 0 else idb, ct)
                reqs.append((rid, mdl, ct))
        srv.step()
        step += 1
    for rid, mdl, ct in reqs:
        out = srv.take(rid)
        assert out is not None, "request not finished"
        mk, keys = (A, ka) if mdl == 0 else (B, kb)
        alone = G.kan_infer(ctx, keys, mk, [ct])
        assert out.level == alone.level
        assert (out.export() == alone.export()).all()
    st = srv.status()
    assert st["active"] == 0 and st["waiting"] == 0


def test_admission_respects_budget(env):
    """Footprints are measured on the device (the pool's used-bytes watermark
    over a probe run of the network): with a budget of 1.5 footprints one
    request runs at a time, the admitted sum and the bytes the device really
    allocated in any step stay within the budget, and a request larger than
    the whole budget is refused instead of being admitted alone."""
    G, ctx, (A, ka, na), _ = env
    one = _req(G, ctx, ka, na, 0, 17)
    probe = G.Server(ctx, 1 << 40)
    fp = probe.footprint(probe.add_model(A, ka))
    # the run needs more than its output ciphertext and less than the
    # hundreds of input-sized buffers a leak would show
    assert one.words() * 8 < fp < 400 * one.words() * 8
    budget = fp + fp // 2
    srv = G.Server(ctx, budget)
    mid = srv.add_model(A, ka)
    assert srv.footprint(mid) == fp  # the same schedule allocates the same bytes
    ids = [srv.submit(mid, _req(G, ctx, ka, na, i, 17)) for i in range(3)]
    for _ in range(20):
        srv.step()
        st = srv.status()
        assert st["active"] <= 1
        assert st["hbm_peak"] <= budget
        assert 0 < st["hbm_measured_peak"] <= budget
    assert all(srv.take(i) is not None for i in ids)
    small = G.Server(ctx, fp // 2)
    m2 = small.add_model(A, ka)
    with pytest.raises(G.CkksError) as e:
        small.submit(m2, one)
    assert e.value.code == -5  # CKKS_ERR_OUT_OF_MEMORY
