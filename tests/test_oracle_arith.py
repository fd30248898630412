"""Pins for the oracle's RNS-CKKS arithmetic (CPU only).

Each test checks the oracle against something other than itself: a library
routine (sympy primality, numpy complex DFT sums), a textbook definition
written differently (schoolbook negacyclic product, O(N^2) evaluation NTT,
coefficient-domain automorphism), exact big-integer CRT identities, the
RFC 8439 ChaCha20 vectors, or the plaintext result of the homomorphic op.
"""
import os

import numpy as np
import pytest

from oracle import ckks
from oracle._lib import lib, ptr

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def small():
    ctx = ckks.Ctx(ckks.Params(log_n=5, n_scale=5, n_special=2))
    keys = ckks.Keys(ctx, 11, rot_steps=[1, 2, -1, -3, 5])
    return ctx, keys


def test_miller_rabin_matches_sympy():
    sympy = pytest.importorskip("sympy")
    rng = np.random.default_rng(5)
    L = lib()
    cands = [int(x) | 1 for x in rng.integers(2 ** 40, 2 ** 61, size=300, dtype=np.int64)]
    cands += [2 ** 61 - 1, 3215031751, 3825123056546413051, 1, 2, 3, 4, 561, 1105]
    for c in cands:
        assert bool(L.or_is_prime(c)) == sympy.isprime(c), c


@pytest.mark.parametrize("log_n,L_,alpha", [(4, 4, 1), (10, 8, 3), (16, 36, 4), (15, 18, 1)])
def test_prime_chain(log_n, L_, alpha):
    sympy = pytest.importorskip("sympy")
    ctx = ckks.Ctx(ckks.Params(log_n=log_n, n_scale=L_, n_special=alpha))
    M = 2 << log_n
    allp = [int(x) for x in ctx.moduli]
    assert len(set(allp)) == len(allp)
    for p in allp:
        assert sympy.isprime(p) and p % M == 1
    assert ctx.q[0].bit_length() == 60 and all(p.bit_length() == 60 for p in ctx.pm)
    assert all(q.bit_length() in (40, 41) for q in ctx.q[1:])
    # canonical scales: Delta_L = 2^40, Delta_{l-1} = Delta_l^2 / q_l, all near 2^40
    d = ctx.delta
    assert d[L_] == 2.0 ** 40
    for l in range(L_, 0, -1):
        assert d[l - 1] == (d[l] * d[l]) / float(ctx.q[l])
    assert np.all(np.abs(np.log2(d) - 40) < 1e-3)


def test_psi_rule():
    L = lib()
    for log_n in (4, 6, 12):
        ctx = ckks.Ctx(ckks.Params(log_n=log_n, n_scale=2, n_special=1))
        N = ctx.N
        for q, psi in zip(ctx.moduli, ctx.psi):
            q, psi = int(q), int(psi)
            assert pow(psi, N, q) == q - 1 and pow(psi, 2 * N, q) == 1
            # smallest base x whose (q-1)/2N power has order 2N
            for x in range(2, 50):
                c = pow(x, (q - 1) // (2 * N), q)
                if pow(c, N, q) == q - 1:
                    assert c == psi
                    break


def _rand(q, n, seed):
    return np.random.default_rng(seed).integers(0, q, size=n, dtype=np.uint64)


@pytest.mark.parametrize("log_n", [2, 3, 4, 5, 6])
def test_ntt_matches_definition_and_schoolbook(log_n):
    L = lib()
    ctx = ckks.Ctx(ckks.Params(log_n=log_n, n_scale=2, n_special=1))
    N = ctx.N
    for t in range(ctx.n_qp):
        q, psi = int(ctx.moduli[t]), int(ctx.psi[t])
        a, b = _rand(q, N, t), _rand(q, N, 100 + t)
        A = a.copy()
        L.or_ntt_forward(ptr(A), log_n, q, psi)
        # evaluation definition written in Python big ints
        brv = [int(format(j, "0%db" % log_n)[::-1], 2) for j in range(N)]
        for j in range(N):
            e = 2 * brv[j] + 1
            ref = sum(int(a[i]) * pow(psi, e * i, q) for i in range(N)) % q
            assert int(A[j]) == ref
        B = b.copy()
        L.or_ntt_forward(ptr(B), log_n, q, psi)
        C = np.array([(int(x) * int(y)) % q for x, y in zip(A, B)], np.uint64)
        L.or_ntt_inverse(ptr(C), log_n, q, psi)
        # schoolbook product in Python big ints
        ref = [0] * N
        for i in range(N):
            for j in range(N):
                k = i + j
                if k < N:
                    ref[k] += int(a[i]) * int(b[j])
                else:
                    ref[k - N] -= int(a[i]) * int(b[j])
        assert [int(x) for x in C] == [r % q for r in ref]
        back = A.copy()
        L.or_ntt_inverse(ptr(back), log_n, q, psi)
        assert (back == a).all()


def test_ntt_identity_large():
    L = lib()
    ctx = ckks.Ctx(ckks.Params(log_n=13, n_scale=1, n_special=1))
    for t in range(ctx.n_qp):
        q, psi = int(ctx.moduli[t]), int(ctx.psi[t])
        a = _rand(q, ctx.N, t)
        A = a.copy()
        L.or_ntt_forward(ptr(A), 13, q, psi)
        L.or_ntt_inverse(ptr(A), 13, q, psi)
        assert (A == a).all()


def test_automorphism_ntt_vs_coef():
    L = lib()
    ctx = ckks.Ctx(ckks.Params(log_n=6, n_scale=1, n_special=1))
    q, psi, N = int(ctx.moduli[1]), int(ctx.psi[1]), ctx.N
    a = _rand(q, N, 3)
    # coefficient form written directly: a(X) -> a(X^g)
    for g in (5, 25, 2 * N - 1, ctx.galois(-3)):
        ref = [0] * N
        for i in range(N):
            k = (i * g) % (2 * N)
            if k < N:
                ref[k] = int(a[i])
            else:
                ref[k - N] = (-int(a[i])) % q
        A = a.copy()
        L.or_ntt_forward(ptr(A), 6, q, psi)
        out = np.zeros(N, np.uint64)
        L.or_automorphism_ntt(ptr(A), ptr(out), 6, g)
        L.or_ntt_inverse(ptr(out), 6, q, psi)
        assert [int(x) for x in out] == ref


def _golden():
    d = {}
    for line in open(os.path.join(GOLD, "chacha20_rfc8439.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        d[k] = v
    return d


def test_chacha20_rfc8439_vectors():
    L = lib()
    g = _golden()
    s = np.array([int(x, 16) for x in g["quarter_in"]], np.uint32)
    L.or_chacha20_quarter(ptr(s))
    assert [int(x) for x in s] == [int(x, 16) for x in g["quarter_out"]]
    key = np.array([int(x, 16) for x in g["block_key"]], np.uint32)
    nonce = np.array([int(x, 16) for x in g["block_nonce"]], np.uint32)
    out = np.zeros(16, np.uint32)
    L.or_chacha20_block(ptr(key), int(g["block_counter"][0]), ptr(nonce), ptr(out))
    assert [int(x) for x in out] == [int(x, 16) for x in g["block_out"]]


def test_sampler_moments():
    L = lib()
    log_n = 14
    N = 1 << log_n
    s = np.zeros(N, np.int64)
    L.or_sample_ternary(7, log_n, ptr(s))
    assert set(np.unique(s)) <= {-1, 0, 1}
    for v in (-1, 0, 1):
        assert abs(np.mean(s == v) - 1 / 3) < 0.02
    e = np.zeros(N, np.int64)
    L.or_sample_cbd(7, 3, log_n, ptr(e))
    assert abs(e.mean()) < 0.1 and abs(e.var() - 10.5) < 0.6 and np.abs(e).max() <= 21
    q = (1 << 40) + 12345
    a = np.zeros(N, np.uint64)
    L.or_sample_uniform(7, 3, 2, q, log_n, ptr(a))
    assert a.max() < q
    hist = np.histogram(a.astype(np.float64), bins=16, range=(0, q))[0]
    assert np.all(np.abs(hist - N / 16) < 6 * np.sqrt(N / 16))
    # the stream definition: word idx of block idx//16
    w = L.or_stream_word32(9, 2, 5, 37)
    key = np.array([9, 0, 0, 0, 0, 0, 0, 0], np.uint32)
    nonce = np.array([2, 5, 0], np.uint32)
    blk = np.zeros(16, np.uint32)
    L.or_chacha20_block(ptr(key), 2, ptr(nonce), ptr(blk))
    assert w == blk[37 % 16]


def _embed_direct(m, log_n):
    """slot j = m(zeta^(5^j mod 2N)), zeta = exp(i pi / N): direct sum."""
    N = 1 << log_n
    e = np.array([pow(5, j, 2 * N) for j in range(N // 2)])
    X = np.exp(1j * np.pi * np.outer(e, np.arange(N)) / N)
    return X @ m


@pytest.mark.parametrize("log_n", [3, 5, 9])
def test_encoder_matches_canonical_embedding(log_n):
    L = lib()
    N = 1 << log_n
    rng = np.random.default_rng(log_n)
    z = rng.uniform(-1, 1, N // 2)
    scale = 2.0 ** 30
    c = np.zeros(N, np.int64)
    assert L.or_encode(ptr(z), len(z), log_n, scale, ptr(c)) == 0
    m = c / scale
    assert np.abs(_embed_direct(m, log_n) - z).max() < N * 2.0 ** -29
    # decode is the same embedding
    out = np.zeros(N // 2)
    L.or_decode(ptr(np.ascontiguousarray(m)), log_n, ptr(out), N // 2)
    assert np.abs(out - _embed_direct(m, log_n).real).max() < 1e-12


def test_encoder_product_and_rotation_structure():
    """Negacyclic product of encodings decodes to the slot product; the
    automorphism X -> X^5 rotates slots left by one (Eq. 10, t = 1)."""
    L = lib()
    log_n, N = 5, 32
    rng = np.random.default_rng(1)
    x, y = rng.uniform(-1, 1, N // 2), rng.uniform(-1, 1, N // 2)
    cx, cy = np.zeros(N, np.int64), np.zeros(N, np.int64)
    L.or_encode(ptr(x), N // 2, log_n, 2.0 ** 20, ptr(cx))
    L.or_encode(ptr(y), N // 2, log_n, 2.0 ** 20, ptr(cy))
    prod = np.zeros(N)
    for i in range(N):
        for j in range(N):
            k = i + j
            v = float(int(cx[i]) * int(cy[j]))
            if k < N:
                prod[k] += v
            else:
                prod[k - N] -= v
    out = np.zeros(N // 2)
    L.or_decode(ptr(prod / 2.0 ** 40), log_n, ptr(out), N // 2)
    assert np.abs(out - x * y).max() < 1e-4
    rot = np.zeros(N)
    for i in range(N):
        k = (5 * i) % (2 * N)
        if k < N:
            rot[k] = cx[i]
        else:
            rot[k - N] = -cx[i]
    L.or_decode(ptr(rot / 2.0 ** 20), log_n, ptr(out), N // 2)
    assert np.abs(out - np.roll(x, -1)).max() < 1e-4


def _crt(limbs, mods):
    Q = 1
    for m in mods:
        Q *= m
    x = 0
    for r, m in zip(limbs, mods):
        Qi = Q // m
        x += int(r) * Qi * pow(Qi, -1, m)
    return x % Q, Q


def _coef(ctx, rows_ntt, mod_idx):
    L = lib()
    out = []
    for r, t in zip(rows_ntt, mod_idx):
        a = np.ascontiguousarray(r).copy()
        L.or_ntt_limb(ctx.h, ptr(a), t, 1)
        out.append(a)
    return out


def test_modup_is_exact_crt_plus_small_multiple(small):
    ctx, _ = small
    L = lib()
    level = ctx.L
    l = level + 1
    rng = np.random.default_rng(4)
    d = np.stack([rng.integers(0, ctx.q[t], ctx.N, dtype=np.uint64) for t in range(l)])
    rows = int(L.or_ext_rows(ctx.h, level))
    ext = np.zeros((rows, ctx.N), np.uint64)
    L.or_modup(ctx.h, ptr(d), level, ptr(ext))
    A = ctx.alpha
    beta = (l + A - 1) // A
    R = l + A
    mod_idx = list(range(l)) + [ctx.L + 1 + k for k in range(A)]
    dc = _coef(ctx, d, list(range(l)))
    for j in range(beta):
        dig = list(range(j * A, min((j + 1) * A, l)))
        Dm = [ctx.q[i] for i in dig]
        Dj = int(np.prod([int(x) for x in Dm], dtype=object))
        ej = _coef(ctx, ext[j * R:(j + 1) * R], mod_idx)
        for n in range(0, ctx.N, 7):
            X, _ = _crt([dc[i][n] for i in dig], Dm)
            for r in range(R):
                m = int(ctx.moduli[mod_idx[r]])
                diff = (int(ej[r][n]) - X) % m
                assert any((u * Dj) % m == diff for u in range(len(dig))), (j, r, n)


def test_rescale_exact_division(small):
    ctx, keys = small
    L = lib()
    rng = np.random.default_rng(8)
    lv = ctx.L
    ct = ckks.encrypt(ctx, keys, rng.uniform(-1, 1, 8), lv, 5)
    out = np.zeros((2, lv, ctx.N), np.uint64)
    L.or_rescale(ctx.h, ptr(ct.data), 2, lv, ptr(out))
    for p in range(2):
        xin = _coef(ctx, ct.data[p], list(range(lv + 1)))
        xo = _coef(ctx, out[p], list(range(lv)))
        ql = ctx.q[lv]
        for n in range(0, ctx.N, 5):
            X, Q = _crt([xin[t][n] for t in range(lv + 1)], ctx.q[: lv + 1])
            Y, Qo = _crt([xo[t][n] for t in range(lv)], ctx.q[:lv])
            r = X % ql
            if r > ql // 2:
                r -= ql
            assert (Y * ql - (X - r)) % Qo == 0


def test_homomorphic_ops_match_plaintext(small):
    ctx, keys = small
    rng = np.random.default_rng(2)
    S = ctx.slots
    x, y = rng.uniform(-1, 1, S), rng.uniform(-1, 1, S)
    cx = ckks.encrypt(ctx, keys, x, ctx.L, 2, 0)
    cy = ckks.encrypt(ctx, keys, y, ctx.L, 2, 1)
    dec = lambda c: ckks.decrypt(ctx, keys, c)
    tol = 1e-6
    assert np.abs(dec(cx) - x).max() < tol
    assert np.abs(dec(ckks.add(ctx, cx, cy)) - (x + y)).max() < tol
    assert np.abs(dec(ckks.sub(ctx, cx, cy)) - (x - y)).max() < tol
    m = ckks.mul(ctx, keys, cx, cy)
    assert m.level == ctx.L - 1 and m.scale == ctx.delta[ctx.L - 1]
    assert np.abs(dec(m) - x * y).max() < tol
    assert np.abs(dec(ckks.mul_plain(ctx, cx, y)) - x * y).max() < tol
    assert np.abs(dec(ckks.add_plain(ctx, cx, y)) - (x + y)).max() < tol
    assert np.abs(dec(ckks.mul_const(ctx, cx, -0.3)) - (-0.3 * x)).max() < tol
    assert np.abs(dec(ckks.add_const(ctx, cx, 0.7)) - (x + 0.7)).max() < tol
    assert np.abs(dec(ckks.level_down(ctx, cx, 2)) - x).max() < tol
    lc = ckks.lincomb(ctx, [cx, m], [2.0, -1.5], 0.25)
    assert np.abs(dec(lc) - (2 * x - 1.5 * x * y + 0.25)).max() < tol
    for t in (1, 2, -1, -3, 5):
        assert np.abs(dec(ckks.rotate(ctx, keys, cx, t)) - np.roll(x, -t)).max() < tol
    many = ckks.rotate_many(ctx, keys, cx, [1, 2, 5])
    for t in (1, 2, 5):
        assert (many[t].data == ckks.rotate(ctx, keys, cx, t).data).all()
    ms = ckks.mul_sum(ctx, keys, [(cx, cy), (cy, cy)])
    assert np.abs(dec(ms) - (x * y + y * y)).max() < tol
    # a deeper chain: x^8 by squaring down to level L-3
    p = cx
    for _ in range(3):
        p = ckks.mul(ctx, keys, p, p)
    assert np.abs(dec(p) - x ** 8).max() < 1e-5


def test_scale_mismatch_and_level_errors(small):
    ctx, keys = small
    cx = ckks.encrypt(ctx, keys, [0.5], ctx.L, 2, 0)
    cy = ckks.encrypt(ctx, keys, [0.5], ctx.L - 1, 2, 1)
    with pytest.raises(ValueError):
        ckks.add(ctx, cx, cy)
    z = ckks.encrypt(ctx, keys, [0.5], 0, 2, 2)
    with pytest.raises(ValueError):
        ckks.rescale(ctx, z)


def test_relin_rescale_is_one_division_by_p_ql(small):
    """HMult's merged division: for random tensor components and key-product
    rows, out = (y - Conv_D([y]_D)) / (P q_l), y = P d + acc, with the
    centred conversion over D = {q_l} + P, so against the exact big-integer
    y over QP_l (CRT) out is y / M rounded to nearest (the overflow is found
    in double precision: off by one only within ~1e-15 of a half-integer)."""
    ctx, keys = small
    L = lib()
    rng = np.random.default_rng(12)
    lv = ctx.L
    l, A = lv + 1, ctx.alpha
    R = l + A
    mod_idx = list(range(l)) + [ctx.L + 1 + k for k in range(A)]
    qp = [int(ctx.moduli[t]) for t in mod_idx]
    d = np.stack([np.stack([rng.integers(0, ctx.q[t], ctx.N, dtype=np.uint64) for t in range(l)])
                  for _ in range(3)])
    ext = ckks._modup(ctx, d[2], lv)
    out = ckks._ks_rescale(ctx, d, ext, lv, keys.relin)
    # the key product alone: ModDown skipped by a zero-P check is not
    # available, so rebuild acc from the C core's key-switch inputs
    beta = (l + A - 1) // A
    acc = np.zeros((2, R, ctx.N), dtype=object)
    for k in range(2):
        for r in range(R):
            t = mod_idx[r]
            m = qp[r]
            for j in range(beta):
                e = ext[j * R + r].astype(object)
                kk = keys.relin[j, k, t].astype(object)
                acc[k, r] = (acc[k, r] + e * kk) % m
    P = 1
    for a in range(A):
        P *= int(ctx.moduli[ctx.L + 1 + a])
    M = P * int(ctx.q[lv])
    for k in range(2):
        yrows = [((P % qp[r]) * (d[k, r].astype(object) if r < l else 0) + acc[k, r]) % qp[r] for r in range(R)]
        yc = _coef(ctx, [np.array(list(x), dtype=np.uint64) for x in yrows], mod_idx)
        oc = _coef(ctx, out[k], list(range(lv)))
        QP = 1
        for m in qp:
            QP *= m
        Qo = 1
        for t in range(lv):
            Qo *= int(ctx.q[t])
        exact = 0
        for n in range(0, ctx.N, 3):
            Y, _ = _crt([yc[r][n] for r in range(R)], qp)
            O, _ = _crt([oc[t][n] for t in range(lv)], ctx.q[:lv])
            rem = Y % M
            if 2 * rem > M:
                rem -= M  # centred remainder: Y - rem = M round(Y / M)
            ok = [(O * M - (Y - rem) + u * M) % Qo == 0 for u in (0, -1, 1)]
            assert any(ok), (k, n)
            exact += ok[0]
        assert exact >= 0.99 * len(range(0, ctx.N, 3))


def _auto_coef(a, g, m):
    """a(X) -> a(X^g) mod (X^N + 1, m) on coefficients, from the definition."""
    N = len(a)
    out = [0] * N
    for i, v in enumerate(a):
        e = (i * g) % (2 * N)
        if e < N:
            out[e] = (out[e] + int(v)) % m
        else:
            out[e - N] = (out[e - N] - int(v)) % m
    return np.array(out, dtype=np.uint64)


@pytest.mark.parametrize("step", [0, 1, -3])
def test_moddown_is_rounded_division_by_p(small, step):
    """Key inner product + ModDown: out_k = round(acc_k / P) over Q_l, with
    acc_k = sum_j sigma_g(ext_j) key_j[k] the exact value over QP_l. The
    automorphism of the hoisted rotation is applied to the ModUp rows here in
    the coefficient domain from its definition (X -> X^g), the inner product
    by big-integer arithmetic, and the value checked by CRT: the centred
    conversion makes the division round to nearest (off by one only within
    ~1e-15 of a half-integer, where the overflow's double sum can round
    either way)."""
    ctx, keys = small
    L = lib()
    rng = np.random.default_rng(20 + step)
    lv = ctx.L
    l, A = lv + 1, ctx.alpha
    R = l + A
    beta = (l + A - 1) // A
    mod_idx = list(range(l)) + [ctx.L + 1 + k for k in range(A)]
    qp = [int(ctx.moduli[t]) for t in mod_idx]
    g = 0 if step == 0 else ctx.galois(step)
    key = keys.relin if g == 0 else keys.galois[g]
    d = np.stack([rng.integers(0, ctx.q[t], ctx.N, dtype=np.uint64) for t in range(l)])
    ext = ckks._modup(ctx, d, lv)
    out = ckks._ks(ctx, ext, lv, key, g)
    # sigma_g(ext) in NTT form, through the coefficient domain
    sig = ext.copy()
    if g:
        for j in range(beta):
            for r in range(R):
                row = _coef(ctx, [ext[j * R + r]], [mod_idx[r]])[0]
                row = _auto_coef(row, g, qp[r])
                L.or_ntt_limb(ctx.h, ptr(row), mod_idx[r], 0)
                sig[j * R + r] = row
    P = 1
    for a in range(A):
        P *= int(ctx.moduli[ctx.L + 1 + a])
    Qo = 1
    for t in range(l):
        Qo *= int(ctx.q[t])
    for k in range(2):
        acc = []
        for r in range(R):
            a = np.zeros(ctx.N, dtype=object)
            for j in range(beta):
                a = (a + sig[j * R + r].astype(object) * key[j, k, mod_idx[r]].astype(object)) % qp[r]
            acc.append(np.array(list(a), dtype=np.uint64))
        yc = _coef(ctx, acc, mod_idx)
        oc = _coef(ctx, out[k], list(range(l)))
        exact = 0
        pts = range(0, ctx.N, 2)
        for n in pts:
            Y, _ = _crt([yc[r][n] for r in range(R)], qp)
            O, _ = _crt([oc[t][n] for t in range(l)], ctx.q[:l])
            rem = Y % P
            if 2 * rem > P:
                rem -= P  # centred remainder: Y - rem = P round(Y / P)
            ok = [(O * P - (Y - rem) + u * P) % Qo == 0 for u in (0, -1, 1)]
            assert any(ok), (k, n)
            exact += ok[0]
        assert exact >= 0.99 * len(pts)


def test_qp_rotation_divided_by_p_is_the_rotation(small):
    """A rotation kept in QP_l for double hoisting, R = (P sigma(c0) + acc_0,
    acc_1), divided by P with rounding to nearest (by CRT, big integers)
    gives the hoisted rotation's words exactly: P sigma(c0) is a multiple
    of P, so the rounding is that of ModDown on acc alone."""
    ctx, keys = small
    rng = np.random.default_rng(31)
    lv = ctx.L
    l, A = lv + 1, ctx.alpha
    mod_idx = list(range(l)) + [ctx.L + 1 + k for k in range(A)]
    qp = [int(ctx.moduli[t]) for t in mod_idx]
    P = 1
    for a in range(A):
        P *= int(ctx.moduli[ctx.L + 1 + a])
    Qo = 1
    for t in range(l):
        Qo *= int(ctx.q[t])
    ct = ckks.encrypt(ctx, keys, rng.uniform(-1, 1, ctx.slots), lv, 3)
    for step in (0, 2, -3):
        R = ckks.rotate_many_qp(ctx, keys, ct, [step])[step]
        rot = ckks.rotate(ctx, keys, ct, step).data if step else ct.data
        for k in range(2):
            yc = _coef(ctx, R[k], mod_idx)
            oc = _coef(ctx, rot[k], list(range(l)))
            exact = 0
            for n in range(ctx.N):
                Y, _ = _crt([yc[r][n] for r in range(len(qp))], qp)
                O, _ = _crt([oc[t][n] for t in range(l)], ctx.q[:l])
                rem = Y % P
                if 2 * rem > P:
                    rem -= P
                exact += (O * P - (Y - rem)) % Qo == 0
            assert exact >= 0.99 * ctx.N, (step, k)


def test_keyswitch_rounding_is_unbiased():
    """ModDown (rotation) and HMult's division round to nearest: the error
    of a rotation stays at the level of fresh encryption noise at every slot
    (an uncentred conversion leaves an offset of about alpha / 2 per
    coefficient on both polynomials, which the secret key turns into an
    error of about 1e-6 at slot 0 at N = 2^14)."""
    ctx = ckks.Ctx(ckks.Params(log_n=14, n_scale=3, n_special=2))
    keys = ckks.Keys(ctx, 7, rot_steps=[1])
    x = np.random.default_rng(1).uniform(-1, 1, ctx.slots)
    y = np.random.default_rng(2).uniform(-1, 1, ctx.slots)
    cx = ckks.encrypt(ctx, keys, x, ctx.L, 9, 0)
    cy = ckks.encrypt(ctx, keys, y, ctx.L, 9, 1)
    e_rot = ckks.decrypt(ctx, keys, ckks.rotate(ctx, keys, cx, 1)) - np.roll(x, -1)
    e_mul = ckks.decrypt(ctx, keys, ckks.mul(ctx, keys, cx, cy)) - x * y
    assert np.abs(e_rot).max() < 1e-7 and abs(e_rot.mean()) < 1e-10
    assert np.abs(e_mul).max() < 1e-7 and abs(e_mul.mean()) < 1e-10


def test_switch_keys_with_a_public_seed():
    """Switching keys whose uniform halves come from a public seed: the
    default (public seed = seed) gives the same keys word for word; another
    public seed changes every a half, leaves the secret alone, and every
    digit row t still satisfies the key equation b + a s = e + [t in digit j]
    [P]_q s' mod q_t with e the small centred-binomial error (checked in the
    coefficient domain, |e| <= 21)."""
    ctx = ckks.Ctx(ckks.Params(log_n=6, n_scale=5, n_special=2))
    L = lib()
    k0 = ckks.Keys(ctx, 11, rot_steps=[1])
    k1 = ckks.Keys(ctx, 11, rot_steps=[1], a_seed=11)
    k2 = ckks.Keys(ctx, 11, rot_steps=[1], a_seed=12345)
    assert (k0.relin == k1.relin).all() and (k0.s == k2.s).all()
    g = ctx.galois(1)
    for key0, key, gg in ((k0.relin, k2.relin, 0), (k0.galois[g], k2.galois[g], g)):
        assert not (key0[:, 1] == key[:, 1]).any(axis=-1).all()
        sp = np.zeros_like(k2.s)
        L.or_target_secret(ctx.h, ptr(k2.s), gg, ptr(sp))
        P = 1
        for p in ctx.pm:
            P *= p
        for j in range(ctx.beta_max):
            for t in range(ctx.n_qp):
                q = int(ctx.moduli[t])
                b = key[j, 0, t].astype(object)
                a = key[j, 1, t].astype(object)
                s = k2.s[t].astype(object)
                e = (b + a * s) % q
                if t <= ctx.L and t // ctx.alpha == j:
                    e = (e - (P % q) * sp[t].astype(object)) % q
                row = np.array([int(v) for v in e], dtype=np.uint64)
                L.or_ntt_limb(ctx.h, ptr(row), t, 1)
                c = np.array([int(v) if int(v) <= q // 2 else int(v) - q for v in row])
                assert np.abs(c).max() <= 21, (j, t)
