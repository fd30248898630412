"""GPU parity of the encrypted KAN layer and network: the CUDA schedule's
ciphertexts must equal the oracle's word for word (same seeded keys,
inputs and model), and decryptions must match the HE-friendly FP64 KAN
within CKKS noise. Sizes: a tiny model at N = 2^7 (several BSGS tiles, ragged
n_i), and the [4,8,4,1] G=5 k=3 network with the full 36-level chain at
N = 2^11, batched at uneven levels."""
import numpy as np
import pytest

from oracle import calibrate, ckks as O, kan_he, kan_plain
from paper_2409_07751_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2409_07751_gb300 import build, ckks
    build.build()
    return ckks


def _setup(G, log_n, L, alpha, model):
    gctx = G.Context(log_n, L, alpha)
    octx = O.Ctx(O.Params(log_n, L, alpha))
    gm = G.Model(gctx, model)
    rots = kan_he.model_rotations(model, octx.slots)
    assert gm.rotations() == rots
    gk = G.Keys(gctx, W.SEED_KEYS, rots)
    ok = O.Keys(octx, W.SEED_KEYS, rots)
    return gctx, octx, gm, gk, ok


def test_tiny_layer_and_network_bit_exact(G):
    model = W.make_model("t", widths=[3, 5, 2], G=3, k=2)
    X = W.uniform_inputs(64, 3)
    m = calibrate.calibrate(model, X, 7, [1])
    gctx, octx, gm, gk, ok = _setup(G, 7, 17, 2, m)
    for li in range(len(m)):
        assert gm.layer_depth(li) == 7
    x = X[:2]
    oc = O.encrypt(octx, ok, x[0], octx.L, W.SEED_ENC, 0)
    gc = G.Ciphertext.import_(gctx, oc.data, oc.level, oc.scale)
    # one layer
    o1 = kan_he.layer_eval(octx, ok, oc, m[0])
    g1 = G.kan_layer_eval(gctx, gk, gm, 0, gc)
    assert g1.level == o1.level and g1.scale == o1.scale
    assert (g1.export()[0] == o1.data).all()
    # whole network through the client path (GPU encryption)
    gin = G.encrypt(gctx, gk, x, octx.L, W.SEED_ENC, 0)
    gout = G.kan_infer(gctx, gk, gm, [gin])
    for b in range(2):
        oc = O.encrypt(octx, ok, x[b], octx.L, W.SEED_ENC, b)
        oo = kan_he.infer(octx, ok, oc, m)
        assert (gout.export()[b] == oo.data).all()
    dec = G.decrypt(gctx, gk, gout, 2)
    hef = kan_plain.forward(m, x, "poly", "poly")
    assert np.abs(dec - hef).max() < 1e-6


@pytest.mark.parametrize("G_,k_", [(1, 0), (2, 1), (4, 0)])
def test_degenerate_grids_bit_exact(G, G_, k_):
    """Order-0 splines (no recursion), a single interval, linear splines."""
    model = W.make_model("t", widths=[3, 2], G=G_, k=k_)
    X = W.uniform_inputs(64, 3)
    m = calibrate.calibrate(model, X, 5, [1])
    gctx, octx, gm, gk, ok = _setup(G, 7, 12, 2, m)
    oc = O.encrypt(octx, ok, X[0], octx.L, W.SEED_ENC, 0)
    gc = G.Ciphertext.import_(gctx, oc.data, oc.level, oc.scale)
    oo = kan_he.infer(octx, ok, oc, m)
    go = G.kan_infer(gctx, gk, gm, [gc])
    assert (go.export()[0] == oo.data).all()
    hef = kan_plain.forward(m, X[:1], "poly", "poly")
    assert np.abs(G.decrypt(gctx, gk, go, 2) - hef).max() < 1e-5


def test_wide_first_layer_chunks_bit_exact(G):
    """40 inputs with G=3, k=2 at N=2^7: 40 * 8 > 64 slots, so the input is
    split into 5 ciphertexts of 8 (request-major batch) and the partial
    outputs are summed."""
    model = W.make_model("t", widths=[40, 4, 2], G=3, k=2)
    X = W.uniform_inputs(64, 40)
    m = calibrate.calibrate(model, X, 7, [1])
    gctx, octx, gm, gk, ok = _setup(G, 7, 17, 2, m)
    K, n_c = kan_he.chunking(m[0], octx.slots)
    assert (K, n_c) == (5, 8)
    outs = []
    batch = []
    for b in range(2):
        xp = np.pad(X[b], (0, K * n_c - 40))
        chunks = [O.encrypt(octx, ok, xp[c * n_c:(c + 1) * n_c], octx.L, W.SEED_ENC, b * K + c)
                  for c in range(K)]
        outs.append(kan_he.infer(octx, ok, chunks, m))
        batch += [xp[c * n_c:(c + 1) * n_c] for c in range(K)]
    gin = G.encrypt(gctx, gk, np.array(batch), octx.L, W.SEED_ENC, 0)
    gout = G.kan_infer(gctx, gk, gm, [gin])
    assert gout.batch == 2
    for b in range(2):
        assert (gout.export()[b] == outs[b].data).all()
    dec = G.decrypt(gctx, gk, gout, 2)
    assert np.abs(dec - kan_plain.forward(m, X[:2], "poly", "poly")).max() < 1e-5


def test_naive_permutation_method_bit_exact(G):
    """The naive method (HE permutation of the basis by P, then W'), on a
    network and on a chunked wide first layer, equals the oracle word for
    word and is one level deeper per layer than lazy combination."""
    model = W.make_model("t", widths=[40, 4, 2], G=3, k=2)
    X = W.uniform_inputs(64, 40)
    m = calibrate.calibrate(model, X, 7, [1])
    naive = [dict(L, naive=True) for L in m]
    gctx, octx, gm, gk, ok = _setup(G, 7, 19, 2, naive)
    lazy = G.Model(gctx, m)
    for li in range(2):
        assert gm.layer_depth(li) == lazy.layer_depth(li) + 1
    K, n_c = kan_he.chunking(m[0], octx.slots)
    xp = np.pad(X[0], (0, K * n_c - 40))
    rows = [xp[c * n_c:(c + 1) * n_c] for c in range(K)]
    chunks = [O.encrypt(octx, ok, r, octx.L, W.SEED_ENC, c) for c, r in enumerate(rows)]
    oo = kan_he.infer(octx, ok, chunks, naive)
    gin = G.encrypt(gctx, gk, np.array(rows), octx.L, W.SEED_ENC, 0)
    go = G.kan_infer(gctx, gk, gm, [gin])
    assert (go.export()[0] == oo.data).all()
    hef = kan_plain.forward(m, X[:1], "poly", "poly")
    assert np.abs(G.decrypt(gctx, gk, go, 2) - hef).max() < 1e-5


@pytest.mark.parametrize("log_n", [8, 13])
def test_graph_replay_matches_eager(G, log_n):
    """With graphs on, the first call of a shape runs eagerly, the second
    captures, the third replays: every result equals the eager schedule's
    word for word, and the replay counts the same kernel launches."""
    model = W.make_model("kan_4_8_4_1")
    X = W.uniform_inputs(256, 4)
    m = calibrate.calibrate(model, X, 27, [3])
    ctx = G.Context(log_n, 36, 4)
    gm = G.Model(ctx, m)
    keys = G.Keys(ctx, W.SEED_KEYS, gm.rotations())
    x = G.encrypt(ctx, keys, X[:3], 36, W.SEED_ENC, 0)
    ref = G.kan_infer(ctx, keys, gm, [x]).export()
    c0 = ctx.launch_counts()
    G.kan_infer(ctx, keys, gm, [x]).close()
    c1 = ctx.launch_counts()
    eager = {k: c1[k] - c0[k] for k in c1 if k != "copy"}
    gm.set_graphs(True)
    for prof in (False, True):  # a profiled capture records its events as graph nodes
        ctx.profile(prof)
        for call in range(3):
            if call == 2:
                ctx.profile_collect()  # keep the replay's records only
            a = ctx.launch_counts()
            out = G.kan_infer(ctx, keys, gm, [x])
            b = ctx.launch_counts()
            assert (out.export() == ref).all(), (prof, call)
            assert {k: b[k] - a[k] for k in b if k != "copy"} == eager, (prof, call)
        if prof:
            p = ctx.profile_collect()
            assert {k: v[2] for k, v in p.items() if k != "copy"} == {k: v for k, v in eager.items() if v}
            assert all(v[0] > 0 for k, v in p.items())
    ctx.profile(False)
    gm.set_graphs(False)
    assert (G.kan_infer(ctx, keys, gm, [x]).export() == ref).all()


def test_level_exhausted_is_an_error(G):
    model = W.make_model("t", widths=[3, 2], G=3, k=2)
    m = calibrate.calibrate(model, W.uniform_inputs(64, 3), 7, [1])
    gctx = G.Context(7, 17, 2)
    gm = G.Model(gctx, m)
    gk = G.Keys(gctx, 1, gm.rotations())
    c = G.encrypt(gctx, gk, [0.1, 0.2, 0.3], 4, seed=1)  # below the layer depth
    with pytest.raises(G.CkksError) as e:
        G.kan_infer(gctx, gk, gm, [c])
    assert e.value.code == -2
    with pytest.raises(G.CkksError):
        G.kan_infer(gctx, gk, gm, [])
    # a hidden layer wider than the slots allow cannot be split by the server
    wide = calibrate.calibrate(W.make_model("t", widths=[3, 40, 2], G=3, k=2),
                               W.uniform_inputs(64, 3), 7, [1])
    with pytest.raises(G.CkksError) as e:
        G.Model(gctx, wide)
    assert e.value.code == -9 and "hidden layer" in str(e.value)


def test_kan_4_8_4_1_batched_uneven_levels(G):
    model = W.make_model("kan_4_8_4_1")
    X = W.uniform_inputs(256, 4)
    m = calibrate.calibrate(model, X, 27, [3])
    gctx, octx, gm, gk, ok = _setup(G, 11, 36, 4, m)
    depth = sum(gm.layer_depth(i) for i in range(3))
    assert depth <= 36
    slack = 36 - depth
    x = X[:3]
    levels = [36, 36 - slack, 36 - min(1, slack)]
    gins = [G.encrypt(gctx, gk, x[b], levels[b], W.SEED_ENC, b) for b in range(3)]
    gout = G.kan_infer(gctx, gk, gm, gins)
    assert gout.batch == 3
    data = gout.export()
    lv = min(levels)
    for b in (0, 1):
        oc = O.encrypt(octx, ok, x[b], levels[b], W.SEED_ENC, b)
        oc = O.level_down(octx, oc, lv)
        oo = kan_he.infer(octx, ok, oc, m)
        assert (data[b] == oo.data).all(), b
    dec = G.decrypt(gctx, gk, gout, 1)
    hef = kan_plain.forward(m, x, "poly", "poly")
    assert np.abs(dec - hef).max() < 1e-4


@pytest.mark.parametrize("b0,G_,k_", [("difference", 3, 2), ("product", 3, 2), ("difference", 4, 0),
                                      ("difference", 2, 1)])
def test_minimax_composite_and_b0_forms_bit_exact(G, b0, G_, k_):
    """PolyComp by a minimax composite (degree 7 then 15, eps = 0.1) and
    either order-0 form of Algorithm 2: one layer and the whole network equal
    the oracle word for word; the difference form is one level shallower per
    layer; decryptions match the HE-friendly FP64 KAN."""
    from oracle import polycomp
    stages, _ = polycomp.composite(0.1, (7, 15))
    model = [dict(L, b0=b0) for L in W.make_model("t", widths=[3, 5, 2], G=G_, k=k_)]
    X = W.uniform_inputs(64, 3)
    m = calibrate.calibrate(model, X, 7, stages)
    gctx, octx, gm, gk, ok = _setup(G, 7, 26, 2, m)
    prod = G.Model(gctx, [dict(L, b0="product") for L in m])
    for li in range(len(m)):
        assert gm.layer_depth(li) == prod.layer_depth(li) - (1 if b0 == "difference" else 0)
    oc = O.encrypt(octx, ok, X[0], octx.L, W.SEED_ENC, 0)
    gc = G.Ciphertext.import_(gctx, oc.data, oc.level, oc.scale)
    o1 = kan_he.layer_eval(octx, ok, oc, m[0])
    g1 = G.kan_layer_eval(gctx, gk, gm, 0, gc)
    assert g1.level == o1.level and g1.scale == o1.scale
    assert (g1.export()[0] == o1.data).all()
    gin = G.encrypt(gctx, gk, X[:2], octx.L, W.SEED_ENC, 0)
    gout = G.kan_infer(gctx, gk, gm, [gin])
    for b in range(2):
        oo = kan_he.infer(octx, ok, O.encrypt(octx, ok, X[b], octx.L, W.SEED_ENC, b), m)
        assert (gout.export()[b] == oo.data).all()
    hef = kan_plain.forward(m, X[:2], "poly", "poly")
    assert np.abs(G.decrypt(gctx, gk, gout, 2) - hef).max() < 1e-5


def test_mixed_level_batch_equals_each_alone(G):
    """kan_infer on inputs at four different levels (one handle each): the
    batch is brought to the lowest level and run together; every output
    equals, word for word, that input brought down to the same level
    (ckks_level_down) and run alone, and equals the oracle."""
    model = W.make_model("t", widths=[3, 5, 2], G=3, k=2)
    X = W.uniform_inputs(64, 3)
    m = calibrate.calibrate(model, X, 7, [1])
    gctx, octx, gm, gk, ok = _setup(G, 7, 20, 2, m)
    levels = [20, 19, 17, 16]
    cts = [G.encrypt(gctx, gk, X[b], lv, W.SEED_ENC, b) for b, lv in enumerate(levels)]
    out = G.kan_infer(gctx, gk, gm, cts)
    assert out.batch == 4
    got = out.export()
    low = min(levels)
    for b, ct in enumerate(cts):
        alone = G.kan_infer(gctx, gk, gm, [G.level_down(gctx, ct, low)])
        assert alone.level == out.level
        assert (alone.export()[0] == got[b]).all(), b
        oc = O.level_down(octx, O.encrypt(octx, ok, X[b], levels[b], W.SEED_ENC, b), low)
        assert (got[b] == kan_he.infer(octx, ok, oc, m).data).all(), b


@pytest.mark.parametrize("b0", ["product", "difference"])
def test_double_hoisted_bsgs_bit_exact(G, b0):
    """Double-hoisted BSGS (baby steps kept in QP_l, one division by P q_l
    per giant step): a layer and the network equal the oracle's double-hoisted
    schedule word for word, decrypt like the hoisted form, and the words
    differ from it (a different rounding)."""
    model = [dict(L, bsgs="double", b0=b0) for L in W.make_model("t", widths=[3, 5, 2], G=3, k=2)]
    X = W.uniform_inputs(64, 3)
    m = calibrate.calibrate(model, X, 7, [1])
    gctx, octx, gm, gk, ok = _setup(G, 7, 17, 2, m)
    single = G.Model(gctx, [dict(L, bsgs="single") for L in m])
    oc = O.encrypt(octx, ok, X[0], octx.L, W.SEED_ENC, 0)
    gc = G.Ciphertext.import_(gctx, oc.data, oc.level, oc.scale)
    o1 = kan_he.layer_eval(octx, ok, oc, m[0])
    g1 = G.kan_layer_eval(gctx, gk, gm, 0, gc)
    assert g1.level == o1.level and g1.scale == o1.scale
    assert (g1.export()[0] == o1.data).all()
    gin = G.encrypt(gctx, gk, X[:2], octx.L, W.SEED_ENC, 0)
    gout = G.kan_infer(gctx, gk, gm, [gin])
    sout = G.kan_infer(gctx, gk, single, [gin])
    for b in range(2):
        oo = kan_he.infer(octx, ok, O.encrypt(octx, ok, X[b], octx.L, W.SEED_ENC, b), m)
        assert (gout.export()[b] == oo.data).all()
    assert not (gout.export() == sout.export()).all()
    hef = kan_plain.forward(m, X[:2], "poly", "poly")
    dd, ds = G.decrypt(gctx, gk, gout, 2), G.decrypt(gctx, gk, sout, 2)
    assert np.abs(dd - hef).max() < 1e-5 and np.abs(dd - ds).max() < 1e-5
