"""Seed-compressed switching keys on the GPU: keys drawn with a public seed
equal the oracle's word for word; compressing them halves the switching
keys' device bytes, and every operation that switches keys (HMult,
hoisted rotations, a KAN inference with double-hoisted BSGS, a bootstrap)
gives the uncompressed keys' ciphertexts word for word, at N = 2^7 and at
N = 2^13 (the clustered transforms)."""
import numpy as np
import pytest

from oracle import ckks as O

pytestmark = pytest.mark.gpu

SEED, PUB = 21, 0x5EED


@pytest.fixture(scope="module")
def G():
    from paper_2409_07751_gb300 import build, ckks
    build.build()
    return ckks


@pytest.mark.parametrize("log_n,L,alpha", [(7, 8, 2), (13, 12, 3)])
def test_public_seed_keys_match_the_oracle_and_compress(G, log_n, L, alpha):
    gctx = G.Context(log_n, L, alpha)
    octx = O.Ctx(O.Params(log_n, L, alpha))
    steps = [1, 3, -2]
    gk = G.Keys(gctx, SEED, steps, public_seed=PUB)
    ok = O.Keys(octx, SEED, steps, a_seed=PUB)
    g1 = octx.galois(1)
    assert (gk.export_switch(0) == ok.relin).all()
    assert (gk.export_switch(g1) == ok.galois[g1]).all()
    full = G.Keys(gctx, SEED, steps, public_seed=PUB)
    before = full.nbytes()
    full.compress()
    after = full.nbytes()
    secret = gctx.n_qp * gctx.N * 8
    assert after - secret == (before - secret) // 2
    assert (full.export_switch(0) == ok.relin).all()  # regenerated
    assert (full.export_switch(g1) == ok.galois[g1]).all()
    rng = np.random.default_rng(3)
    x = G.encrypt(gctx, gk, rng.uniform(-1, 1, (3, gctx.slots)), L, 5, 0)
    prod = [G.mul(gctx, k, x, x).export() for k in (gk, full)]
    rots = [[r.export() for r in G.rotate_hoisted(gctx, k, x, steps)] for k in (gk, full)]
    assert (prod[0] == prod[1]).all()
    assert all((u == v).all() for u, v in zip(*rots))
    plain = G.Keys(gctx, SEED, steps)  # no public seed: refused
    with pytest.raises(G.CkksError):
        plain.compress()


def test_compressed_keys_kan_and_bootstrap_bit_exact(G):
    from oracle import calibrate, kan_he
    from paper_2409_07751_gb300 import workloads as W
    # a KAN [3,4,2] with double-hoisted BSGS
    model = [dict(L, bsgs="double") for L in W.make_model("t", widths=[3, 4, 2], G=3, k=2)]
    X = W.uniform_inputs(64, 3)
    m = calibrate.calibrate(model, X, 7, [1])
    gctx = G.Context(7, 17, 2)
    gm = G.Model(gctx, m)
    rots = kan_he.model_rotations(m, gctx.slots)
    a = G.Keys(gctx, SEED, rots, public_seed=PUB)
    b = G.Keys(gctx, SEED, rots, public_seed=PUB)
    b.compress()
    x = G.encrypt(gctx, a, X[:2], 17, W.SEED_ENC, 0)
    assert (G.kan_infer(gctx, a, gm, [x]).export() == G.kan_infer(gctx, b, gm, [x]).export()).all()
    # one bootstrap (double-hoisted transforms, conjugation key)
    gctx = G.Context(7, 24, 2, q0_bits=60, scale_bits=50)
    gp = G.BootPlan(gctx, 6, 127, 2, 2)
    a = G.Keys(gctx, SEED, gp.rotations(), hamming_weight=16, conjugation=True, public_seed=PUB)
    b = G.Keys(gctx, SEED, gp.rotations(), hamming_weight=16, conjugation=True, public_seed=PUB)
    b.compress()
    z = np.linspace(-1, 1, gctx.slots)
    ct = G.encrypt(gctx, a, z, 0, 3, 0)
    ra, rb = gp.bootstrap(a, ct), gp.bootstrap(b, ct)
    assert (ra.export() == rb.export()).all()
    assert np.abs(G.decrypt(gctx, b, rb, gctx.slots)[0] - z).max() < 1e-6
