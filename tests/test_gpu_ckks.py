"""GPU parity of the RNS-CKKS core: every ciphertext, key and NTT word the
CUDA library produces must equal the oracle's (bit-exact integer work), and
decryptions must agree to the FP64 decoder's rounding.

Parameter sets span the single-CTA NTT (N <= 4096) and the two-phase NTT
(N = 2^13 .. 2^16, column factors 2 .. 16), hybrid digits with a ragged last
digit, and alpha = 1 (one special prime)."""
import numpy as np
import pytest

from oracle import ckks as O

pytestmark = pytest.mark.gpu

PARAMS = {
    "n32": dict(log_n=5, n_scale=5, n_special=2),
    "n4k": dict(log_n=12, n_scale=4, n_special=3),
    "n8k": dict(log_n=13, n_scale=3, n_special=1),
    "n16k": dict(log_n=14, n_scale=3, n_special=2),
    "n32k": dict(log_n=15, n_scale=4, n_special=1),
    "n64k": dict(log_n=16, n_scale=3, n_special=2),
    # the digit layout the autotuner picks within log2 QP <= 1740 at N = 2^16
    "n64k_a5": dict(log_n=16, n_scale=6, n_special=5, p_bits=48),
}


@pytest.fixture(scope="module")
def G():
    from paper_2409_07751_gb300 import build, ckks
    build.build()
    return ckks


_cache = {}


def pair(G, name, steps=(1, -1, 3, -5)):
    if name not in _cache:
        p = PARAMS[name]
        pb = p.get("p_bits", 60)
        gctx = G.Context(p["log_n"], p["n_scale"], p["n_special"], p_bits=pb)
        octx = O.Ctx(O.Params(p["log_n"], p["n_scale"], p["n_special"], p_bits=pb))
        gk = G.Keys(gctx, 7, steps)
        ok = O.Keys(octx, 7, steps)
        _cache[name] = (gctx, octx, gk, ok)
    return _cache[name]


@pytest.mark.parametrize("name", list(PARAMS))
def test_context_matches_oracle(G, name):
    p = PARAMS[name]
    pb = p.get("p_bits", 60)
    gctx = G.Context(p["log_n"], p["n_scale"], p["n_special"], p_bits=pb)
    octx = O.Ctx(O.Params(p["log_n"], p["n_scale"], p["n_special"], p_bits=pb))
    assert (gctx.moduli == octx.moduli).all()
    assert (gctx.delta == octx.delta).all()
    gctx.close()


@pytest.mark.parametrize("log_n", [4, 5, 8, 12, 13, 14, 15, 16])
def test_ntt_bit_exact(G, log_n):
    import torch
    gctx = G.Context(log_n, 3, 2)
    octx = O.Ctx(O.Params(log_n, 3, 2))
    rows, limbs = 7, 4  # ragged: 7 rows over 4 moduli
    rng = np.random.default_rng(log_n)
    a = np.stack([rng.integers(0, int(gctx.moduli[r % limbs]), 1 << log_n, dtype=np.uint64) for r in range(rows)])
    d = torch.from_numpy(a.view(np.int64).copy()).cuda()
    gctx.ntt(d.data_ptr(), rows, limbs)
    gctx.synchronize()
    f = d.cpu().numpy().view(np.uint64)
    ref = a.copy()
    for r in range(rows):
        octx.L_.or_ntt_limb(octx.h, ref[r].ctypes.data, r % limbs, 0)
    assert (f == ref).all()
    gctx.ntt(d.data_ptr(), rows, limbs, inverse=True)
    gctx.synchronize()
    assert (d.cpu().numpy().view(np.uint64) == a).all()
    gctx.close()


@pytest.mark.parametrize("name", ["n32", "n4k", "n8k"])
def test_keys_bit_exact(G, name):
    gctx, octx, gk, ok = pair(G, name)
    assert (gk.export_secret() == ok.s).all()
    assert (gk.export_switch(0) == ok.relin).all()
    for g, key in ok.galois.items():
        assert (gk.export_switch(g) == key).all()


@pytest.mark.parametrize("name", ["n32", "n4k", "n8k", "n64k"])
def test_encrypt_decrypt(G, name):
    gctx, octx, gk, ok = pair(G, name)
    rng = np.random.default_rng(3)
    v = rng.uniform(-1, 1, (3, min(gctx.slots, 100)))
    for lv in (gctx.L, 1):
        gct = G.encrypt(gctx, gk, v, lv, seed=5, first_index=10)
        data = gct.export()
        for b in range(3):
            oct_ = O.encrypt(octx, ok, v[b], lv, 5, 10 + b)
            assert (data[b] == oct_.data).all()
            assert gct.scale == oct_.scale
        dec = G.decrypt(gctx, gk, gct, v.shape[1])
        assert np.abs(dec - v).max() < 1e-6
        assert (dec[0] == O.decrypt(octx, ok, O.Ct(data[0], lv, gct.scale), v.shape[1])).all()


def _both(G, gctx, octx, gk, ok, lv, seed, idx):
    rng = np.random.default_rng(seed)
    v = rng.uniform(-1, 1, gctx.slots)
    oc = O.encrypt(octx, ok, v, lv, 9, idx)
    gc = G.Ciphertext.import_(gctx, oc.data, lv, oc.scale)
    return v, oc, gc


def _same(gc, oc):
    assert gc.level == oc.level
    assert gc.scale == oc.scale
    assert (gc.export()[0] == oc.data).all()


@pytest.mark.parametrize("name", ["n32", "n4k", "n8k", "n16k", "n32k", "n64k", "n64k_a5"])
def test_ops_bit_exact(G, name):
    gctx, octx, gk, ok = pair(G, name)
    L = gctx.L
    x, ox, gx = _both(G, gctx, octx, gk, ok, L, 1, 0)
    y, oy, gy = _both(G, gctx, octx, gk, ok, L, 2, 1)
    _same(G.add(gctx, gx, gy), O.add(octx, ox, oy))
    _same(G.sub(gctx, gx, gy), O.sub(octx, ox, oy))
    _same(G.mul_relin(gctx, gk, gx, gy), O.mul_relin(octx, ok, ox, oy))
    _same(G.rescale(gctx, gx), O.rescale(octx, ox))
    m = G.mul(gctx, gk, gx, gy)
    om = O.mul(octx, ok, ox, oy)
    _same(m, om)
    _same(G.mul_plain(gctx, gx, y), O.mul_plain(octx, ox, y))
    _same(G.add_plain(gctx, gx, y), O.add_plain(octx, ox, y))
    _same(G.mul_const(gctx, gx, -0.37), O.mul_const(octx, ox, -0.37))
    _same(G.add_const(gctx, gx, 0.61), O.add_const(octx, ox, 0.61))
    _same(G.level_down(gctx, gx, 1), O.level_down(octx, ox, 1))
    _same(G.mul(gctx, gk, gx, m), O.mul(octx, ok, ox, om))  # mixed levels
    for t in (1, -1, 3, -5):
        _same(G.rotate(gctx, gk, gx, t), O.rotate(octx, ok, ox, t))
    hs = G.rotate_hoisted(gctx, gk, gx, [1, 3, -5])
    for h, t in zip(hs, [1, 3, -5]):
        _same(h, O.rotate(octx, ok, ox, t))
    dec = G.decrypt(gctx, gk, m)[0]
    assert np.abs(dec - x * y).max() < 1e-6


@pytest.mark.parametrize("name", ["n16k", "n64k"])
def test_unfused_form_matches_oracle(G, name):
    """With kernel fusion off (separate conversion, transform and pointwise
    launches) every op still equals the oracle word for word."""
    gctx, octx, gk, ok = pair(G, name)
    gctx.set_fusion(False)
    try:
        L = gctx.L
        x, ox, gx = _both(G, gctx, octx, gk, ok, L, 1, 0)
        y, oy, gy = _both(G, gctx, octx, gk, ok, L, 2, 1)
        _same(G.mul(gctx, gk, gx, gy), O.mul(octx, ok, ox, oy))
        _same(G.rescale(gctx, gx), O.rescale(octx, ox))
        _same(G.level_down(gctx, gx, 1), O.level_down(octx, ox, 1))
        _same(G.rotate(gctx, gk, gx, 3), O.rotate(octx, ok, ox, 3))
        for h, t in zip(G.rotate_hoisted(gctx, gk, gx, [1, -5]), [1, -5]):
            _same(h, O.rotate(octx, ok, ox, t))
    finally:
        gctx.set_fusion(True)


def test_batched_ops_match_single(G):
    gctx, octx, gk, ok = pair(G, "n4k")
    rng = np.random.default_rng(11)
    v = rng.uniform(-1, 1, (4, 64))
    w = rng.uniform(-1, 1, (4, 64))
    a = G.encrypt(gctx, gk, v, gctx.L, seed=1)
    b = G.encrypt(gctx, gk, w, gctx.L, seed=2)
    m = G.mul(gctx, gk, a, b)
    r = G.rotate(gctx, gk, m, 1)
    data = r.export()
    for i in range(4):
        ai, bi = a.slice(i, 1), b.slice(i, 1)
        ri = G.rotate(gctx, gk, G.mul(gctx, gk, ai, bi), 1)
        assert (ri.export()[0] == data[i]).all()
    dec = G.decrypt(gctx, gk, r, 63)
    assert np.abs(dec - (v * w)[:, 1:64]).max() < 1e-6


def test_errors(G):
    gctx, octx, gk, ok = pair(G, "n32")
    a = G.encrypt(gctx, gk, [0.5], gctx.L, seed=1)
    b = G.encrypt(gctx, gk, [0.5], gctx.L - 1, seed=1)
    with pytest.raises(G.CkksError) as e:
        G.add(gctx, a, b)
    assert e.value.code == -2
    with pytest.raises(G.CkksError) as e:
        G.rotate(gctx, gk, a, 2)
    assert e.value.code == -4
    z = G.encrypt(gctx, gk, [0.5], 0, seed=1)
    with pytest.raises(G.CkksError) as e:
        G.rescale(gctx, z)
    assert e.value.code == -2
    with pytest.raises(G.CkksError) as e:
        G.encrypt(gctx, gk, [1e12], gctx.L, seed=1)
    assert e.value.code == -7


def test_autotune_keyswitch_layout(G):
    """The autotuner times only layouts within the log2 QP bound whose special
    modulus covers the largest digit, and returns the fastest of them."""
    alpha, p_bits, tried = G.autotune_keyswitch(16, 36, 1740, batch=2)
    assert alpha in tried and len(tried) >= 3 and 1 not in tried  # alpha = 1: 37 digits
    assert tried[alpha] == min(tried.values())
    for a in tried:
        p = min(60, (1740 - 60 - 36 * 40) // a)
        assert p >= 30 and a * p >= 60 + (a - 1) * 40
    assert p_bits == min(60, (1740 - 60 - 36 * 40) // alpha)
    print("digit layouts (alpha: ms per HMult+HRot, batch 2):", tried)


def test_async_import_is_ordered_before_later_work(G):
    """ckks_ct_import_async copies on a caller stream; the library's stream
    waits for the copy, so an op issued right after sees the imported words."""
    import torch
    gctx, octx, gk, ok = pair(G, "n64k")
    x, ox, gx = _both(G, gctx, octx, gk, ok, gctx.L, 1, 0)
    host = torch.from_numpy(ox.data.view(np.int64).copy()).pin_memory()
    cs = torch.cuda.Stream()
    c = G.Ciphertext.import_from_async(gctx, host.data_ptr(), 1, gctx.L, ox.scale, cs.cuda_stream)
    _same(G.rescale(gctx, c), O.rescale(octx, ox))
    assert (c.export()[0] == ox.data).all()


def test_staged_inner_product_batch_over_stages(G):
    """A batch of 7 runs the TMA-staged key inner product through every
    stage more than once (three stages, so each mbarrier completes two or
    three phases); HMult and hoisted rotations of all 7 equal the oracle."""
    gctx, octx, gk, ok = pair(G, "n8k")
    rng = np.random.default_rng(21)
    L = gctx.L
    ocs = [O.encrypt(octx, ok, rng.uniform(-1, 1, gctx.slots), L, 3, i) for i in range(7)]
    data = np.stack([o.data for o in ocs])
    g = G.Ciphertext.import_(gctx, data, L, ocs[0].scale)
    md = G.mul(gctx, gk, g, g).export()
    rs = [h.export() for h in G.rotate_hoisted(gctx, gk, g, [1, -5])]
    for i, o in enumerate(ocs):
        assert (md[i] == O.mul(octx, ok, o, o).data).all(), i
        assert (rs[0][i] == O.rotate(octx, ok, o, 1).data).all(), i
        assert (rs[1][i] == O.rotate(octx, ok, o, -5).data).all(), i


def test_bounded_wait_reports_timeout_and_context_survives(G):
    """A device wait that cannot complete runs out after its cycle limit, the
    kernel returns, the host reads CKKS_ERR_TIMEOUT once, and the context
    keeps computing bit-exact results."""
    gctx, octx, gk, ok = pair(G, "n4k")
    assert gctx.selftest_wait(1 << 20) == -8
    gctx.synchronize()  # the status word was cleared by the report
    x, ox, gx = _both(G, gctx, octx, gk, ok, gctx.L, 4, 0)
    _same(G.rotate(gctx, gk, gx, 1), O.rotate(octx, ok, ox, 1))
    gctx.synchronize()
