"""Pins for the oracle's CKKS bootstrapping (CPU only, N = 2^7).

Each step is checked against what the mathematics fixes rather than against
itself: the decoding matrix against the canonical embedding (odd powers of a
primitive 2N-th root of unity), the factored transforms against that matrix
and its inverse (numpy), merged levels against their stages, the monomial
product against multiplication by i, ModRaise against the exact
big-integer identity t = m + q0 I with the Hamming-weight bound on I, the
conjugation and the dense transform against numpy's complex arithmetic on
the slots, the modular-reduction interpolant against m / Delta (closed form
of the scaled sine), and the whole pipeline against the slots it started
from.
"""
import math

import numpy as np
import pytest

from oracle import boot, ckks

H = 16  # Hamming weight of the sparse secret


def _setup(q0_bits, scale_bits=40, K=4, levels=(2, 2)):
    ctx = ckks.Ctx(ckks.Params(log_n=7, n_scale=24, n_special=2, q0_bits=q0_bits,
                               scale_bits=scale_bits))
    plan = boot.Plan(ctx, K, 127, *levels)
    lt_steps = [7, 14, 21, 57]  # the generic transform test's rotations
    return ctx, boot.BootKeys(ctx, 7, plan.steps(ctx) + lt_steps, h=H), plan


@pytest.fixture(scope="module")
def c20():
    """q0 / Delta = 2^20, the gap of the configurations' chains."""
    return _setup(60, levels=(3, 3))


@pytest.fixture(scope="module")
def c10():
    return _setup(50)


@pytest.fixture(scope="module")
def s50():
    """50-bit scale primes under a 60-bit q0: a bootstrappable chain."""
    return _setup(60, scale_bits=50)


@pytest.fixture(scope="module")
def s50d(s50):
    """The same keys with double-hoisted transforms."""
    ctx, keys, plan = s50
    return ctx, keys, boot.Plan(ctx, plan.K, plan.degree, len(plan.cts), len(plan.stc), "double")


def _complex_ct(ctx, keys, z, level):
    """A ciphertext at `level` whose slots are the complex z: Re z encrypted,
    times the plaintext z / Re z, rescaled."""
    re = np.where(np.abs(z.real) < 0.3, 0.3, z.real)
    ct = ckks.encrypt(ctx, keys, re, level + 1, 5)
    S = ckks.plain_scale(ctx, ct.scale, level + 1)
    pt = boot.encode_complex(ctx, z / re, level + 1, S)
    prod = np.zeros_like(ct.data)
    ctx.L_.or_mul_plain(ctx.h, boot.ptr(ct.data), boot.ptr(pt), 2, level + 2, boot.ptr(prod))
    return ckks.rescale(ctx, ckks.Ct(prod, level + 1, ct.scale * S))


def test_sparse_secret_has_weight_h(c20):
    ctx, keys, _ = c20
    s = keys.s_coef
    assert np.count_nonzero(s) == H
    assert set(np.unique(s[s != 0]).tolist()) <= {-1, 1}
    s2 = np.zeros(ctx.N, np.int64)
    ctx.L_.or_sample_sparse_ternary(8, ctx.log_n, H, boot.ptr(s2))
    assert np.count_nonzero(s2) == H and not np.array_equal(s, s2)


def test_decode_matrix_is_canonical_embedding(c20):
    ctx, _, _ = c20
    N, n = ctx.N, ctx.slots
    E = boot.decode_matrix(ctx)
    zeta = E[:, 1]
    # X^i decodes to the i-th powers of the slots' roots
    for i in (0, 2, 3, 17, N - 1):
        assert np.abs(E[:, i] - zeta ** i).max() < 1e-12
    # the roots with their conjugates are exactly the primitive 2N-th roots
    ang = np.angle(np.concatenate([zeta, zeta.conj()])) / np.pi * N  # odd integers mod 2N
    k = np.mod(np.rint(ang).astype(int), 2 * N)
    assert np.abs(np.abs(zeta) - 1).max() < 1e-12
    assert sorted(k.tolist()) == list(range(1, 2 * N, 2))
    assert len(set(np.rint(ang[:n]).astype(int).tolist())) == n


def _dense(n, d):
    M = np.zeros((n, n), complex)
    for o, v in d.items():
        M[np.arange(n), (np.arange(n) + o) % n] += v
    return M


def _bitrev(n):
    b = n.bit_length() - 1
    P = np.zeros((n, n))
    for i in range(n):
        P[int(format(i, "0%db" % b)[::-1], 2), i] = 1
    return P


def test_special_fft_factors_the_decoding_map(c20):
    ctx, _, _ = c20
    n = ctx.slots
    log_n = n.bit_length() - 1
    E = boot.decode_matrix(ctx)
    U = E[:, :n]
    assert np.abs(E[:, n:] - 1j * U).max() < 1e-12  # zeta_j^n = i: z = U (t_lo + i t_hi)
    F, Fi = np.eye(n), np.eye(n)
    for s in range(1, log_n + 1):
        F = _dense(n, boot.fft_stage(ctx, s)) @ F
    for s in range(log_n, 0, -1):
        Fi = _dense(n, boot.fft_stage(ctx, s, inverse=True)) @ Fi
    BR = _bitrev(n)
    assert np.abs(F @ BR - U).max() < 1e-12
    assert np.abs(Fi - n * BR @ np.linalg.inv(U)).max() < 1e-11
    rng = np.random.default_rng(2)
    z = rng.normal(size=n) + 1j * rng.normal(size=n)
    for n_levels in (1, 2, 3, log_n):
        for inverse, want in ((False, F @ z), (True, Fi @ z)):
            lts = boot.transform_levels(ctx, n_levels, inverse)
            assert len(lts) == n_levels
            w = z
            for lt in lts:
                assert len(lt.diags) <= 2 * n
                w = lt.matrix_apply(w)
            assert np.abs(w - want).max() < 1e-11 * np.abs(want).max()


@pytest.mark.parametrize("form", ["single", "double"])
def test_linear_transform_matches_numpy(c20, form):
    ctx, keys, _ = c20
    rng = np.random.default_rng(7)
    n = ctx.slots
    diags = [(rng.normal(size=n) + 1j * rng.normal(size=n)) / 3 for _ in range(7)]
    diags[4][:] = 0  # skipped
    lt = boot.LinearTransform(-7, 7, diags, g1=4, form=form)  # offsets -7, 0, ..., 35
    assert lt.steps(n) == [7, 14, 21, 57]  # baby 7, 14, 21; giant -7 = 57 and 21
    z = rng.uniform(-1, 1, n) + 1j * rng.uniform(-1, 1, n)
    ct = _complex_ct(ctx, keys, z, 12)
    out = boot.linear_transform(ctx, keys, ct, lt)
    assert out.level == 11
    assert np.abs(boot.decrypt_crt(ctx, keys, out) - lt.matrix_apply(z)).max() < 1e-6


def test_monomial_and_wide_constant(c20):
    ctx, keys, _ = c20
    rng = np.random.default_rng(9)
    z = rng.uniform(-1, 1, ctx.slots) + 1j * rng.uniform(-1, 1, ctx.slots)
    ct = _complex_ct(ctx, keys, z, 10)
    for k, f in ((ctx.N // 2, 1j), (3 * ctx.N // 2, -1j), (ctx.N, -1), (1, None)):
        got = boot.decrypt_crt(ctx, keys, boot.mul_monomial(ctx, ct, k))
        if f is None:  # X multiplies slot j by zeta_j = E[j, 1]
            f = boot.decode_matrix(ctx)[:, 1]
        assert np.abs(got - f * z).max() < 1e-6
    big = ckks.encrypt(ctx, keys, rng.uniform(-1, 1, ctx.slots) * 2.0 ** 20, 12, 4)
    vals = boot.decrypt_crt(ctx, keys, big).real
    out = boot.mul_const_wide(ctx, big, 2.0 ** -30)
    assert out.level == 10 and abs(out.scale / ctx.delta[10] - 1) < 2 ** -30
    assert np.abs(boot.decrypt_crt(ctx, keys, out).real - vals * 2.0 ** -30).max() < 1e-10


def test_mod_raise_adds_a_small_multiple_of_q0(c20):
    ctx, keys, _ = c20
    z = np.random.default_rng(4).uniform(-1, 1, ctx.slots)
    ct = ckks.encrypt(ctx, keys, z, 0, 9)
    raised = boot.mod_raise(ctx, ct)
    assert raised.level == ctx.L
    assert np.array_equal(raised.data[:, 0], ct.data[:, 0])
    q0 = ctx.q[0]
    m = boot.decrypt_coeffs_crt(ctx, keys, ct)  # centred mod q0
    t = boot.decrypt_coeffs_crt(ctx, keys, raised)
    I = [(ti - mi) // q0 for ti, mi in zip(t, m)]
    assert all((ti - mi) % q0 == 0 for ti, mi in zip(t, m))
    # |c0 + c1 s| <= (h + 1) q0 / 2 with centred c0, c1 and h entries of s
    assert max(abs(i) for i in I) <= (H + 1) // 2 + 1
    assert any(i != 0 for i in I)  # the overflow is really there


def test_conjugation_conjugates_the_slots(c20):
    ctx, keys, _ = c20
    rng = np.random.default_rng(6)
    z = rng.uniform(-1, 1, ctx.slots) + 1j * rng.uniform(-1, 1, ctx.slots)
    ct = _complex_ct(ctx, keys, z, 10)
    assert np.abs(boot.decrypt_crt(ctx, keys, ct) - z).max() < 1e-6
    cj = boot.conjugate(ctx, keys, ct)
    assert np.abs(boot.decrypt_crt(ctx, keys, cj) - z.conj()).max() < 1e-6


def test_coeff_to_slot_gives_the_scaled_coefficients(c20):
    ctx, keys, plan = c20
    n = ctx.slots
    z = np.random.default_rng(8).uniform(-1, 1, n)
    raised = boot.mod_raise(ctx, ckks.encrypt(ctx, keys, z, 0, 10))
    t = np.array([float(x) for x in boot.decrypt_coeffs_crt(ctx, keys, raised)])
    y = t / (raised.scale * 2.0 ** boot.mod_exponent(ctx, plan.K))
    assert np.abs(y).max() <= 1.0
    lo, hi = boot.coeff_to_slot(ctx, keys, raised, plan.K, plan.cts)
    br = _bitrev(n).argmax(axis=1)  # slot p holds coefficient brv(p)
    for ct, want in ((lo, y[:n][br]), (hi, y[n:][br])):
        got = boot.decrypt_crt(ctx, keys, ct)
        assert np.abs(got.real - want).max() < 1e-9
        assert np.abs(got.imag).max() < 1e-9


@pytest.mark.parametrize("q0_bits,bound", [(60, 1e-8), (50, 1e-9)])
def test_eval_mod_interpolant_reduces_mod_q0(q0_bits, bound):
    ctx = ckks.Ctx(ckks.Params(log_n=7, n_scale=20, n_special=2, q0_bits=q0_bits))
    K, deg = 4, 127
    coeffs = boot.eval_mod_coeffs(ctx, K, deg)
    q0, D = float(ctx.q[0]), float(ctx.delta[0])
    e = boot.mod_exponent(ctx, K)
    assert 2.0 ** e >= (K + 1) * q0 / D > 2.0 ** (e - 1)
    c = q0 / D
    mD = np.linspace(-1, 1, 201)
    # c / (2 pi) sin(2 pi x / c) = x - (2 pi / c)^2 x^3 / 6 + ...
    sine_err = (2 * math.pi / c) ** 2 / 6 * np.abs(mD) ** 3
    for I in range(-K, K + 1):
        y = (mD * D + q0 * I) / (D * 2.0 ** e)
        got = np.polynomial.chebyshev.chebval(y, coeffs)
        assert (np.abs(got - mD) <= sine_err * 1.001 + bound).all(), I


@pytest.mark.parametrize("fx,bound", [("c20", 2e-2), ("c10", 1e-4), ("s50", 1e-6), ("s50d", 1e-6)])
def test_bootstrap_restores_the_slots(fx, bound, request):
    """Precision follows q0 / Delta and the scale: EvalMod multiplies the
    noise of y by about 2^e ~ (K + 1) q0 / Delta, so 40-bit scale primes
    under a 60-bit q0 (the configurations' chains) leave a few 1e-3, a
    50-bit q0 a few 1e-6 and 50-bit scale primes under a 60-bit q0 1e-7."""
    ctx, keys, plan = request.getfixturevalue(fx)
    z = np.random.default_rng(1).uniform(-1, 1, ctx.slots)
    ct = ckks.encrypt(ctx, keys, z, 0, 3)
    out = boot.bootstrap(ctx, keys, ct, plan)
    assert out.level >= 8
    got = boot.decrypt_crt(ctx, keys, out)
    assert np.abs(got.real - z).max() < bound
    assert np.abs(got.imag).max() < bound
    sq = ckks.mul(ctx, keys, out, out)  # the refreshed levels are usable
    assert np.abs(ckks.decrypt(ctx, keys, sq) - z * z).max() < 3 * bound


def test_stage_roots_are_correctly_rounded():
    """The transforms' roots of unity (the 2^17-th roots) equal mpmath's
    50-digit cos and sin rounded to double, bit for bit, at a spread of
    indices in every octant: the plan's diagonals are the same on every
    machine."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    cs, sn = boot._root_table(boot.ROOT_LOG)
    M = 1 << boot.ROOT_LOG
    for k in list(range(1, M, 997)) + [M // 8, 3 * M // 8, M - 1]:
        t = 2 * mpmath.pi * k / M
        assert cs[k] == float(mpmath.cos(t)) and sn[k] == float(mpmath.sin(t)), k
    for q, (c, s_) in enumerate(((1, 0), (0, 1), (-1, 0), (0, -1))):  # quarter turns exactly
        assert cs[q * M // 4] == c and sn[q * M // 4] == s_


@pytest.mark.parametrize("count", [1, 3, 4, 7])
def test_pack_and_unpack_trees(count):
    """The packed refresh's rotation trees on encrypted vectors: pack_tree
    puts ciphertext b's block [0, nb) at slots [b nb, b nb + nb) (numpy
    concatenation, the rest zero), and unpack_tree returns rot(packed, b nb)
    for every b (numpy roll), for a ragged and a power-of-two count."""
    ctx = ckks.Ctx(ckks.Params(log_n=7, n_scale=6, n_special=2))
    n, nb = ctx.slots, 8
    steps = sorted({(s * nb) % n for s in (1, 2, 4)} | {(-s * nb) % n for s in (1, 2, 4)})
    keys = ckks.Keys(ctx, 3, rot_steps=steps)
    rng = np.random.default_rng(count)
    vals = [np.concatenate([rng.uniform(-1, 1, 5), np.zeros(n - 5)]) for _ in range(count)]
    cts = [ckks.encrypt(ctx, keys, v, 5, 4, b) for b, v in enumerate(vals)]
    packed = boot.pack_tree(ctx, keys, cts, nb)
    want = np.zeros(n)
    for b, v in enumerate(vals):
        want[b * nb:(b + 1) * nb] = v[:nb]
    got = ckks.decrypt(ctx, keys, packed)
    assert np.abs(got - want).max() < 1e-6
    for b, u in enumerate(boot.unpack_tree(ctx, keys, packed, count, nb)):
        assert np.abs(ckks.decrypt(ctx, keys, u) - np.roll(want, -b * nb)).max() < 1e-6
