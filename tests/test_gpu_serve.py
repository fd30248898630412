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


def test_deep_model_served_with_refreshes():
    """A four-layer model of depth 7 per layer on a 24-level chain with a
    bootstrapping plan: the server refreshes a group before the fourth layer
    as kan_infer does. Two requests submitted together share every group
    (packed refresh) and equal kan_infer on the pair word for word; a request
    submitted one step later runs alone (refreshed by itself) and equals
    kan_infer on it alone."""
    from paper_2409_07751_gb300 import build, ckks as G
    from oracle import kan_plain
    build.build()
    ctx = G.Context(7, 24, 2, q0_bits=60, scale_bits=50)
    m = calibrate.calibrate(W.make_model("t", widths=[3, 5, 5, 5, 2], G=3, k=2),
                            W.uniform_inputs(64, 3), 7, [1])
    M = G.Model(ctx, m)
    plan = G.BootPlan(ctx, 6, 127, 2, 2)
    M.set_bootstrap(plan)
    keys = G.Keys(ctx, 7, sorted(set(M.rotations()) | set(plan.rotations()) | set(M.refresh_rotations(2))),
                  hamming_weight=16, conjugation=True)
    X = W.uniform_inputs(3, 3, seed=77)
    cts = [G.encrypt(ctx, keys, X[i], 24, W.SEED_ENC, i) for i in range(3)]
    srv = G.Server(ctx, 1 << 40)
    mid = srv.add_model(M, keys)
    r0, r1 = srv.submit(mid, cts[0]), srv.submit(mid, cts[1])
    srv.step()
    r2 = srv.submit(mid, cts[2])
    for _ in range(6):
        srv.step()
    pair = G.kan_infer(ctx, keys, M, [G.Ciphertext.import_(ctx, np.concatenate(
        [cts[0].export(), cts[1].export()]), 24, cts[0].scale)])
    outs = [srv.take(r) for r in (r0, r1, r2)]
    assert all(o is not None for o in outs)
    assert (outs[0].export()[0] == pair.export()[0]).all()
    assert (outs[1].export()[0] == pair.export()[1]).all()
    alone = G.kan_infer(ctx, keys, M, [cts[2]])
    assert (outs[2].export() == alone.export()).all()
    hef = kan_plain.forward(m, X, "poly", "poly")
    for i, o in enumerate(outs):
        assert np.abs(G.decrypt(ctx, keys, o, 2)[0] - hef[i]).max() < 1e-4
