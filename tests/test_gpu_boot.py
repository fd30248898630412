"""GPU parity of CKKS bootstrapping with the oracle (oracle/boot.py): the
CUDA ModRaise, monomial and wide-constant products, conjugation, slot
linear transforms, CoeffToSlot, EvalMod, SlotToCoeff and the whole refresh
must equal the oracle's ciphertexts word for word (same seeded sparse-secret
keys, input ciphertext, transform diagonals and EvalMod coefficients).
Sizes: N = 2^7 (the small transform kernels; hoisted and double-hoisted
transforms) and N = 2^13 (the clustered transforms, double hoisting, a batch
of 2 against two oracle runs). The library's own plan
(merged diagonals, exponent, Chebyshev coefficients) is checked against the
oracle's by value, and a full-size refresh (N = 2^16, sparse secret of
weight 192) against the slots it started from."""
import numpy as np
import pytest

from oracle import boot as OB, ckks as O

pytestmark = pytest.mark.gpu

SEED = 7
H = 16


@pytest.fixture(scope="module")
def G():
    from paper_2409_07751_gb300 import build, ckks
    build.build()
    return ckks


def _setup(G, log_n, L, alpha, K, degree, levels, extra=(), form="single"):
    params = dict(q0_bits=60, scale_bits=50)
    octx = O.Ctx(O.Params(log_n, L, alpha, **params))
    plan = OB.Plan(octx, K, degree, *levels, form=form)
    steps = sorted(set(plan.steps(octx)) | set(extra))
    okeys = OB.BootKeys(octx, SEED, steps, h=H)
    gctx = G.Context(log_n, L, alpha, **params)
    gkeys = G.Keys(gctx, SEED, steps, hamming_weight=H, conjugation=True)
    return octx, plan, okeys, gctx, gkeys


def _gpu_plan(G, gctx, octx, plan, stc_level):
    cts = [G.LinearTransform(gctx, octx.L - i, lt.base, lt.stride, lt.diags, g1=lt.g1,
                             in_scale=octx.delta[0] if i == 0 else 0.0, form=lt.form)
           for i, lt in enumerate(plan.cts)]
    stc = [G.LinearTransform(gctx, stc_level - i, lt.base, lt.stride, lt.diags, g1=lt.g1,
                             form=lt.form)
           for i, lt in enumerate(plan.stc)]
    return G.BootPlan.from_parts(gctx, OB.mod_exponent(octx, plan.K), plan.cheb, cts, stc)


def _same(g, o, b=0):
    assert g.level == o.level and g.scale == o.scale
    assert (g.export()[b] == o.data).all()


@pytest.fixture(scope="module")
def small(G):
    return _setup(G, 7, 24, 2, 6, 127, (2, 2), extra=(5, 10, 15, 59))


def test_sparse_keys_bit_exact(G, small):
    octx, plan, okeys, gctx, gkeys = small
    assert (gkeys.export_secret() == okeys.s).all()
    assert (gkeys.export_switch(0) == okeys.relin).all()
    g = 2 * octx.N - 1
    assert (gkeys.export_switch(g) == okeys.galois[g]).all()
    g5 = octx.galois(plan.steps(octx)[0])
    assert (gkeys.export_switch(g5) == okeys.galois[g5]).all()


def test_boot_primitives_bit_exact(G, small):
    octx, plan, okeys, gctx, gkeys = small
    z = np.random.default_rng(2).uniform(-1, 1, octx.slots)
    oc = O.encrypt(octx, okeys, z, 0, 3, 0)
    gc = G.Ciphertext.import_(gctx, oc.data, oc.level, oc.scale)
    for level in (octx.L, 5):
        _same(G.mod_raise(gctx, gc, level), OB.mod_raise(octx, oc, level))
    o12 = O.encrypt(octx, okeys, z * 2.0 ** 8, 12, 3, 1)
    g12 = G.Ciphertext.import_(gctx, o12.data, o12.level, o12.scale)
    for k in (1, octx.N // 2, 3 * octx.N // 2, octx.N, 2 * octx.N - 1):
        _same(G.mul_monomial(gctx, g12, k), OB.mul_monomial(octx, o12, k))
    _same(G.conjugate(gctx, gkeys, g12), OB.conjugate(octx, okeys, o12))
    for c in (2.0 ** -25, 3.0 ** -20):
        _same(G.mul_const_wide(gctx, g12, c), OB.mul_const_wide(octx, o12, c))


@pytest.mark.parametrize("form", ["single", "double"])
def test_linear_transform_bit_exact(G, small, form):
    octx, plan, okeys, gctx, gkeys = small
    rng = np.random.default_rng(5)
    n = octx.slots
    diags = [(rng.normal(size=n) + 1j * rng.normal(size=n)) / 3 for _ in range(6)]
    diags[2][:] = 0
    diags[4][:] = 0  # the first diagonal of the second giant step
    lt = OB.LinearTransform(-5, 5, diags, g1=4, form=form)  # offsets -5 .. 20
    glt = G.LinearTransform(gctx, 10, lt.base, lt.stride, lt.diags, g1=lt.g1, form=form)
    assert glt.rotations() == lt.steps(n)
    z = rng.uniform(-1, 1, n)
    oc = O.encrypt(octx, okeys, z, 10, 3, 2)
    gc = G.Ciphertext.import_(gctx, oc.data, oc.level, oc.scale)
    _same(glt.apply(gkeys, gc), OB.linear_transform(octx, okeys, oc, lt))
    with pytest.raises(G.CkksError):
        glt.apply(gkeys, G.Ciphertext.import_(gctx, oc.data[:, :10], 9, octx.delta[9]))


def _stages_bit_exact(G, setup, batch):
    octx, plan, okeys, gctx, gkeys = setup
    rng = np.random.default_rng(11)
    zs = rng.uniform(-1, 1, (batch, octx.slots))
    ocs = [O.encrypt(octx, okeys, zs[b], 0, 3, b) for b in range(batch)]
    gc = G.Ciphertext.import_(gctx, np.stack([c.data for c in ocs]), 0, ocs[0].scale)
    o_raised = [OB.mod_raise(octx, c) for c in ocs]
    o_cts = [OB.coeff_to_slot(octx, okeys, r, plan.K, plan.cts) for r in o_raised]
    o_mod = [(OB.kan_he.eval_cheb(octx, okeys, lo, plan.cheb),
              OB.kan_he.eval_cheb(octx, okeys, hi, plan.cheb)) for lo, hi in o_cts]
    o_out = [OB.slot_to_coeff(octx, okeys, lo, hi, plan.stc) for lo, hi in o_mod]
    gp = _gpu_plan(G, gctx, octx, plan, min(o_mod[0][0].level, o_mod[0][1].level))
    g_raised = G.mod_raise(gctx, gc, octx.L)
    glo, ghi = gp.coeff_to_slot(gkeys, g_raised)
    gmlo, gmhi = gp.eval_mod(gkeys, glo), gp.eval_mod(gkeys, ghi)
    gout = gp.slot_to_coeff(gkeys, gmlo, gmhi)
    gfull = gp.bootstrap(gkeys, gc)
    for b in range(batch):
        _same(g_raised, o_raised[b], b)
        _same(glo, o_cts[b][0], b)
        _same(ghi, o_cts[b][1], b)
        _same(gmlo, o_mod[b][0], b)
        _same(gmhi, o_mod[b][1], b)
        _same(gout, o_out[b], b)
        _same(gfull, o_out[b], b)
    got = G.decrypt(gctx, gkeys, gfull, octx.slots)
    assert np.abs(got - zs).max() < 1e-6


def test_bootstrap_stages_bit_exact_small(G, small):
    _stages_bit_exact(G, small, 1)


def test_bootstrap_stages_bit_exact_small_double_hoisted(G, small):
    octx, plan, okeys, gctx, gkeys = small
    dplan = OB.Plan(octx, plan.K, plan.degree, len(plan.cts), len(plan.stc), form="double")
    _stages_bit_exact(G, (octx, dplan, okeys, gctx, gkeys), 2)


def test_bootstrap_stages_bit_exact_clustered_transforms(G):
    setup = _setup(G, 13, 18, 3, 6, 127, (3, 3), form="double")
    _stages_bit_exact(G, setup, 2)


def test_library_plan_matches_oracle(G, small):
    octx, plan, okeys, gctx, gkeys = small
    for n_levels in (1, 2, 3):
        for inverse in (False, True):
            for i, lt in enumerate(OB.transform_levels(octx, n_levels, inverse)):
                base, stride, d = G.boot_levels(gctx, n_levels, inverse, i)
                assert (base, stride) == (lt.base, lt.stride)
                assert np.abs(d - np.array(lt.diags)).max() < 1e-12
    gp = G.BootPlan(gctx, 6, 127, 2, 2, form="single")
    assert gp.e == OB.mod_exponent(octx, 6) == 13
    assert np.abs(gp.coefficients() - plan.cheb).max() < 1e-9 * np.abs(plan.cheb).max()
    assert gp.cts_level == octx.L
    assert sorted(gp.rotations()) == plan.steps(octx)


def test_library_plan_bootstraps(G, small):
    octx, plan, okeys, gctx, gkeys = small
    gp = G.BootPlan(gctx, 6, 127, 2, 2)  # double hoisting: its own baby-step count
    gkeys = G.Keys(gctx, SEED, gp.rotations(), hamming_weight=H, conjugation=True)
    z = np.random.default_rng(4).uniform(-1, 1, (2, octx.slots))
    gc = G.encrypt(gctx, gkeys, z, 0, 9, 0)
    out = gp.bootstrap(gkeys, gc)
    assert out.level == gp.stc_level - 2
    assert np.abs(G.decrypt(gctx, gkeys, out, octx.slots) - z).max() < 1e-6


def test_bootstrap_full_size(G):
    """N = 2^16, 60-bit q0 under 28 primes of 50 bits, 5 special primes of 60
    bits (log QP = 1760), sparse secret of weight 192 (|I| <= 30: 31 q0 / Delta
    stays below 2^15, so the sine has 32 periods on [-1, 1]), EvalMod of
    degree 255, three merged levels each way, 11 levels left. Precision: every
    rescale at a 2^50 scale leaves about 2^-41.5 in each slot of y; EvalMod
    multiplies it by 2^15 (and the Paterson-Stockmeyer basis by about 13),
    SlotToCoeff sums N/2 such coefficient errors: a few 1e-4 (the oracle at
    N = 2^13 with these parameters: 2.3e-5)."""
    gctx = G.Context(16, 28, 5, q0_bits=60, scale_bits=50)
    gp = G.BootPlan(gctx, 30, 255, 3, 3)
    assert gp.e == 15
    keys = G.Keys(gctx, SEED, gp.rotations(), hamming_weight=192, conjugation=True)
    z = np.random.default_rng(6).uniform(-1, 1, (2, gctx.slots))
    gc = G.encrypt(gctx, keys, z, 0, 9, 0)
    out = gp.bootstrap(keys, gc)
    assert out.level == 11
    err = np.abs(G.decrypt(gctx, keys, out, gctx.slots) - z).max()
    assert err < 1e-3, err
    sq = G.mul(gctx, keys, out, out)
    assert np.abs(G.decrypt(gctx, keys, sq, gctx.slots) - z * z).max() < 3e-3


@pytest.mark.parametrize("batch", [1, 2])
def test_deep_kan_refreshed_between_layers_bit_exact(G, batch):
    """Four layers of depth 7 on a 24-level chain: the library refreshes the
    batch before the fourth layer (levels 24 -> 17 -> 10 -> 3); a batch of
    two is refreshed packed (masked to the 5 output slots, one level, packed
    into one ciphertext, one bootstrap, unpacked: 10 levels after), a single
    ciphertext alone. The outputs equal the oracle's with the same refresh,
    word for word, and the HE-friendly FP64 KAN within 1e-4."""
    from oracle import calibrate, kan_he, kan_plain
    from paper_2409_07751_gb300 import workloads as W
    octx, plan, okeys, gctx, gkeys = _setup(G, 7, 24, 2, 6, 127, (2, 2), form="double")
    model = W.make_model("t", widths=[3, 5, 5, 5, 2], G=3, k=2)
    X = W.uniform_inputs(64, 3)
    m = calibrate.calibrate(model, X, 7, [1])
    gm = G.Model(gctx, m)
    assert [gm.layer_depth(i) for i in range(len(m))] == [7, 7, 7, 7]
    assert gm.refresh_rotations(2) == [8, 56]  # +-8: the block of the 5 output slots
    rots = sorted(set(kan_he.model_rotations(m, octx.slots)) | set(plan.steps(octx))
                  | set(gm.refresh_rotations(batch)))
    okeys = OB.BootKeys(octx, SEED, rots, h=H)
    gkeys = G.Keys(gctx, SEED, rots, hamming_weight=H, conjugation=True)
    probe = OB.kan_he.layer_eval(octx, okeys, O.encrypt(octx, okeys, X[0], octx.L, 1, 0), m[0])
    assert octx.L - probe.level == 7
    x = X[:batch]
    ocs = [O.encrypt(octx, okeys, x[b], octx.L, W.SEED_ENC, b) for b in range(batch)]
    gc = G.Ciphertext.import_(gctx, np.stack([c.data for c in ocs]), octx.L, ocs[0].scale)
    stc_level = octx.L - len(plan.cts) - 2 - 8
    gp = _gpu_plan(G, gctx, octx, plan, stc_level)
    gm.set_bootstrap(gp)
    gout = G.kan_infer(gctx, gkeys, gm, [gc])
    oo = OB.infer_deep(octx, okeys, ocs, m, plan, refresh_before={3}, packed=batch > 1)
    for b in range(batch):
        _same(gout, oo[b], b)
    assert gout.level == stc_level - len(plan.stc) - 7
    hef = kan_plain.forward(m, x, "poly", "poly")
    assert np.abs(G.decrypt(gctx, gkeys, gout, 2) - hef).max() < 1e-4
    with pytest.raises(G.CkksError):  # without the plan the fourth layer runs out of levels
        gm.set_bootstrap(None)
        G.kan_infer(gctx, gkeys, gm, [gc])


def test_deep_kan_full_size(G):
    """A five-layer [4,8,8,8,4,1] KAN (G=5, k=3, SiLU degree 27, the degree-7
    and 15 minimax comparison with eps 0.12 in the difference form: 12
    levels per layer, 60 in all) at N = 2^16 on a 29-level 50-bit chain
    (alpha = 4, log QP = 1750): no leveled chain inside the security budget
    holds it. Two merged CoeffToSlot levels leave 13 levels per refresh (12
    for a layer, one for the packing mask); kan_infer refreshes the batch of
    8 packed before layers 3, 4 and 5. Outputs against the FP64 KAN."""
    from oracle import calibrate, kan_plain, polycomp
    from paper_2409_07751_gb300 import workloads as W
    gctx = G.Context(16, 29, 4, q0_bits=60, scale_bits=50)
    model = [dict(L, b0="difference") for L in W.make_model("t", widths=[4, 8, 8, 8, 4, 1], G=5, k=3)]
    Xcal = W.uniform_inputs(256, 4, seed=W.SEED_INPUTS + 1000)
    m = calibrate.calibrate(model, Xcal, 27, polycomp.composite(0.12, (7, 15))[0])
    gm = G.Model(gctx, m)
    assert [gm.layer_depth(i) for i in range(5)] == [12] * 5
    gp = G.BootPlan(gctx, 30, 255, 2, 3)
    assert gp.stc_level - 3 == 13
    keys = G.Keys(gctx, SEED, sorted(set(gm.rotations()) | set(gp.rotations())
                                     | set(gm.refresh_rotations(8))),
                  hamming_weight=192, conjugation=True)
    gm.set_bootstrap(gp)
    x = W.uniform_inputs(8, 4)
    gc = G.encrypt(gctx, keys, x, 29, W.SEED_ENC, 0)
    out = G.kan_infer(gctx, keys, gm, [gc])
    assert out.level == 1
    dec = G.decrypt(gctx, keys, out, 1)
    hef = kan_plain.forward(m, x, "poly", "poly")
    exact = kan_plain.forward(m, x, "exact", "exact")
    err_hef, err_exact = np.abs(dec - hef).max(), np.abs(dec - exact).max()
    print("deep KAN: vs HE-friendly %.2e, vs exact %.2e" % (err_hef, err_exact))
    assert err_hef < 2e-3, err_hef


def test_entry_points_reject_invalid_input(G, small):
    """The bootstrapping and key entry points refuse what they document as
    invalid (and the context keeps working): ModRaise of a ciphertext above
    level 0, a transform of only zero diagonals, diagonals of the wrong
    width, a plan with K = 0 or a chain too short, a public seed equal to
    the seed; compressing twice is harmless."""
    octx, plan, okeys, gctx, gkeys = small
    z = np.linspace(-1, 1, gctx.slots)
    c3 = G.encrypt(gctx, gkeys, z, 3, 1, 0)
    with pytest.raises(G.CkksError) as e:
        G.mod_raise(gctx, c3, gctx.L)
    assert e.value.code == -2
    zero = G.LinearTransform(gctx, 3, 0, 1, np.zeros((2, gctx.slots)))
    with pytest.raises(G.CkksError):
        zero.apply(gkeys, c3)
    with pytest.raises(ValueError):
        G.LinearTransform(gctx, 3, 0, 1, np.zeros((2, gctx.slots + 1)))
    with pytest.raises(G.CkksError):
        G.BootPlan(gctx, 0, 127, 2, 2)
    short = G.Context(7, 8, 2, q0_bits=60, scale_bits=50)
    with pytest.raises(G.CkksError) as e:
        G.BootPlan(short, 6, 127, 2, 2)  # 17 levels needed
    assert e.value.code == -2
    with pytest.raises(G.CkksError):
        G.Keys(gctx, 5, [1], public_seed=5)
    k = G.Keys(gctx, 5, [1], public_seed=6)
    k.compress()
    k.compress()
    assert np.abs(G.decrypt(gctx, k, G.rotate(gctx, k, G.encrypt(gctx, k, z, 3, 1, 0), 1), gctx.slots)[0]
                  - np.roll(z, -1)).max() < 1e-6
    # the context still computes after the refusals
    out = G.mul(gctx, gkeys, c3, c3)
    assert np.abs(G.decrypt(gctx, gkeys, out, gctx.slots)[0] - z * z).max() < 1e-6
