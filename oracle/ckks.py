"""Oracle RNS-CKKS ciphertext layer (test infrastructure only).

Wraps the C core in `ckks_oracle.c` with level and scale bookkeeping. The
homomorphic operations follow the paper's HE section (Eqs. 6-10): add,
subtract, multiply by ciphertext or plaintext, and rotation, where
rot(x, t) moves slot j+t to slot j (left for t > 0, right for t < 0).

Scale rule (a reading; the paper does not fix one): every ciphertext at
level l carries the canonical scale Delta_l of the prime chain, where
Delta_{l-1} = Delta_l^2 / q_l. Products of two level-l ciphertexts rescale
onto Delta_{l-1}; plaintext operands are encoded at the scale that lands the
rescaled product on the canonical scale; moving a ciphertext to a lower level
multiplies it by an integer constant and rescales.

HMult (a reading; the paper delegates key switching to SEAL): the
relinearisation's ModDown by P and the rescale by q_level are one division
by P q_level with a fast basis conversion of the dropped limbs, so each
product pays one set of forward transforms for both.
"""
import numpy as np

from . import _lib
from ._lib import ptr

SNAP = 2.0 ** -30  # relative distance under which a rescaled scale is canonical


class Params:
    def __init__(self, log_n, n_scale, n_special, q0_bits=60, scale_bits=40, p_bits=60):
        self.log_n = log_n
        self.n_scale = n_scale
        self.n_special = n_special
        self.q0_bits = q0_bits
        self.scale_bits = scale_bits
        self.p_bits = p_bits


class Ctx:
    def __init__(self, params):
        L = _lib.lib()
        self.L_ = L
        self.p = params
        self.h = L.or_ctx_create(params.log_n, params.q0_bits, params.scale_bits,
                                 params.n_scale, params.p_bits, params.n_special)
        if not self.h:
            raise RuntimeError("oracle: prime chain generation failed")
        self.log_n = params.log_n
        self.N = 1 << params.log_n
        self.slots = self.N // 2
        self.L = params.n_scale
        self.alpha = params.n_special
        self.n_qp = self.L + 1 + self.alpha
        self.beta_max = (self.L + 1 + self.alpha - 1) // self.alpha
        self.moduli = np.zeros(self.n_qp, np.uint64)
        self.psi = np.zeros(self.n_qp, np.uint64)
        self.delta = np.zeros(self.L + 1, np.float64)
        L.or_ctx_info(self.h, ptr(self.moduli), ptr(self.psi), ptr(self.delta))
        self.q = [int(x) for x in self.moduli[: self.L + 1]]
        self.pm = [int(x) for x in self.moduli[self.L + 1:]]

    def __del__(self):
        try:
            self.L_.or_ctx_destroy(self.h)
        except Exception:
            pass

    def galois(self, step):
        return int(self.L_.or_galois_elt(self.h, int(step)))


class Keys:
    """Secret key, relinearisation key and Galois keys, all generated from one
    seed; a_seed (optional) draws the switching keys' uniform halves from a
    separate public seed instead."""

    def __init__(self, ctx, seed, rot_steps=(), relin=True, a_seed=None):
        L = ctx.L_
        self.ctx = ctx
        self.seed = seed
        self.a_seed = a_seed
        N = ctx.N
        self.s = np.zeros((ctx.n_qp, N), np.uint64)
        self.s_coef = np.zeros(N, np.int64)
        L.or_keygen_secret(ctx.h, seed, ptr(self.s), ptr(self.s_coef))
        self.relin = self._switch_key(0) if relin else None
        self.galois = {}
        for t in rot_steps:
            g = ctx.galois(t)
            if g != 1 and g not in self.galois:
                self.galois[g] = self._switch_key(g)

    def _switch_key(self, g):
        ctx = self.ctx
        sp = np.zeros_like(self.s)
        ctx.L_.or_target_secret(ctx.h, ptr(self.s), g, ptr(sp))
        key = np.zeros((ctx.beta_max, 2, ctx.n_qp, ctx.N), np.uint64)
        a_seed = getattr(self, "a_seed", None)
        ctx.L_.or_keygen_switch_pub(ctx.h, self.seed, self.seed if a_seed is None else a_seed,
                                    ptr(self.s), ptr(sp), g, ptr(key))
        return key


class Ct:
    """A ciphertext: data[poly][limb][N] in NTT form, level = limbs - 1."""

    def __init__(self, data, level, scale):
        self.data = np.ascontiguousarray(data, dtype=np.uint64)
        self.level = level
        self.scale = float(scale)

    def copy(self):
        return Ct(self.data.copy(), self.level, self.scale)


# ---------------------------------------------------------------- encode / crypt
def encode(ctx, v, level, scale):
    v = np.ascontiguousarray(v, dtype=np.float64)
    pt = np.zeros((level + 1, ctx.N), np.uint64)
    rc = ctx.L_.or_encode_plain(ctx.h, ptr(v), len(v), level, scale, ptr(pt))
    if rc != 0:
        raise OverflowError("oracle: encoding overflow")
    return pt


def encrypt(ctx, keys, v, level, seed, index=0):
    v = np.ascontiguousarray(v, dtype=np.float64)
    ct = np.zeros((2, level + 1, ctx.N), np.uint64)
    rc = ctx.L_.or_encrypt(ctx.h, ptr(keys.s), ptr(v), len(v), level, seed, index, ptr(ct))
    if rc != 0:
        raise OverflowError("oracle: encoding overflow")
    return Ct(ct, level, ctx.delta[level])


def decrypt(ctx, keys, ct, n=None):
    n = ctx.slots if n is None else n
    out = np.zeros(n, np.float64)
    ctx.L_.or_decrypt(ctx.h, ptr(keys.s), ptr(ct.data), ct.level, ct.scale, ptr(out), n)
    return out


# ---------------------------------------------------------------- linear ops
def _check_pair(a, b):
    if a.level != b.level:
        raise ValueError("level mismatch %d vs %d" % (a.level, b.level))
    if abs(a.scale / b.scale - 1.0) > SNAP:
        raise ValueError("scale mismatch %r vs %r" % (a.scale, b.scale))


def add(ctx, a, b):
    _check_pair(a, b)
    out = np.zeros_like(a.data)
    ctx.L_.or_add(ctx.h, ptr(a.data), ptr(b.data), 2, a.level + 1, 0, ptr(out))
    return Ct(out, a.level, a.scale)


def sub(ctx, a, b):
    _check_pair(a, b)
    out = np.zeros_like(a.data)
    ctx.L_.or_add(ctx.h, ptr(a.data), ptr(b.data), 2, a.level + 1, 1, ptr(out))
    return Ct(out, a.level, a.scale)


def mul_int(ctx, a, k):
    out = np.zeros_like(a.data)
    ctx.L_.or_mul_int(ctx.h, ptr(a.data), int(k), 2, a.level + 1, ptr(out))
    return Ct(out, a.level, a.scale)


def round_const(c, scale):
    v = float(np.rint(c * scale))
    if not abs(v) < 9.2e18:
        raise OverflowError("constant too large for its scale")
    return int(v)


def add_const(ctx, a, c):
    """a + c in every slot: c encoded at a's scale (constant polynomial)."""
    out = a.copy()
    ctx.L_.or_add_int(ctx.h, ptr(out.data), round_const(c, a.scale), a.level + 1)
    return out


def add_plain(ctx, a, v):
    """a + v slot-wise, v encoded at a's scale and level."""
    pt = encode(ctx, v, a.level, a.scale)
    out = a.copy()
    ctx.L_.or_add(ctx.h, ptr(a.data[0]), ptr(pt), 1, a.level + 1, 0, ptr(out.data[0]))
    return out


def mod_drop(ctx, a, level):
    if level > a.level:
        raise ValueError("mod_drop cannot raise the level")
    return Ct(a.data[:, : level + 1, :].copy(), level, a.scale)


def rescale(ctx, a):
    if a.level < 1:
        raise ValueError("level exhausted")
    lv = a.level
    out = np.zeros((2, lv, ctx.N), np.uint64)
    ctx.L_.or_rescale(ctx.h, ptr(a.data), 2, lv, ptr(out))
    s = a.scale / ctx.q[lv]
    d = ctx.delta[lv - 1]
    if abs(s / d - 1.0) < SNAP:
        s = d
    return Ct(out, lv - 1, s)


def plain_scale(ctx, ct_scale, level):
    """Scale of a plaintext that, multiplied into a level-`level` operand of
    scale ct_scale and rescaled, lands on Delta_{level-1}."""
    return (ctx.delta[level - 1] * float(ctx.q[level])) / ct_scale


def mul_plain(ctx, a, v):
    """a (x) v slot-wise, then rescale: level-1, canonical scale."""
    S = plain_scale(ctx, a.scale, a.level)
    pt = encode(ctx, v, a.level, S)
    out = np.zeros_like(a.data)
    ctx.L_.or_mul_plain(ctx.h, ptr(a.data), ptr(pt), 2, a.level + 1, ptr(out))
    return rescale(ctx, Ct(out, a.level, a.scale * S))


def mul_const(ctx, a, c):
    """a * c (scalar) then rescale."""
    S = plain_scale(ctx, a.scale, a.level)
    return rescale(ctx, Ct(mul_int(ctx, a, round_const(c, S)).data, a.level, a.scale * S))


def level_down(ctx, a, level):
    """Bring a to `level` with the canonical scale Delta_level."""
    if level == a.level and abs(a.scale / ctx.delta[level] - 1.0) < SNAP:
        return a
    if level >= a.level:
        raise ValueError("level_down needs a lower level")
    b = mod_drop(ctx, a, level + 1)
    S = plain_scale(ctx, b.scale, level + 1)
    return rescale(ctx, Ct(mul_int(ctx, b, round_const(1.0, S)).data, level + 1, b.scale * S))


def lincomb(ctx, cts, coeffs, const=0.0, level=None):
    """sum_i coeffs[i] * cts[i] + const at `level` (default: lowest input level - 1).

    Each term is mod-dropped to level+1 and multiplied by the integer
    rint(c_i * S_i) with S_i = Delta_level * q_{level+1} / scale_i; the sum is
    rescaled once, then `const` is added at Delta_level.
    """
    if level is None:
        level = min(c.level for c in cts) - 1
    top = level + 1
    acc = None
    for ct, c in zip(cts, coeffs):
        if c == 0.0:
            continue
        b = mod_drop(ctx, ct, top)
        S = (ctx.delta[level] * float(ctx.q[top])) / b.scale
        t = mul_int(ctx, b, round_const(c, S))
        if acc is None:
            acc = t.data
        else:
            o = np.zeros_like(acc)
            ctx.L_.or_add(ctx.h, ptr(acc), ptr(t.data), 2, top + 1, 0, ptr(o))
            acc = o
    if acc is None:
        acc = np.zeros((2, top + 1, ctx.N), np.uint64)
    out = rescale(ctx, Ct(acc, top, ctx.delta[level] * float(ctx.q[top])))
    out.scale = ctx.delta[level]
    if const != 0.0:
        out = add_const(ctx, out, const)
    return out


# ---------------------------------------------------------------- key switching
def _modup(ctx, poly, level):
    rows = int(ctx.L_.or_ext_rows(ctx.h, level))
    ext = np.zeros((rows, ctx.N), np.uint64)
    ctx.L_.or_modup(ctx.h, ptr(np.ascontiguousarray(poly)), level, ptr(ext))
    return ext


def _ks(ctx, ext, level, key, g):
    out = np.zeros((2, level + 1, ctx.N), np.uint64)
    ctx.L_.or_keyswitch_ext(ctx.h, ptr(ext), level, ptr(key), g, ptr(out))
    return out


def tensor(ctx, a, b):
    if a.level != b.level:
        raise ValueError("tensor needs equal levels")
    out = np.zeros((3, a.level + 1, ctx.N), np.uint64)
    ctx.L_.or_tensor(ctx.h, ptr(a.data), ptr(b.data), a.level + 1, ptr(out))
    return out


def relinearise(ctx, keys, d, level, scale):
    """(d0, d1, d2) -> (d0, d1) + KeySwitch_{s^2 -> s}(d2)."""
    ext = _modup(ctx, d[2], level)
    o = _ks(ctx, ext, level, keys.relin, 0)
    out = np.zeros((2, level + 1, ctx.N), np.uint64)
    ctx.L_.or_add(ctx.h, ptr(np.ascontiguousarray(d[:2])), ptr(o), 2, level + 1, 0, ptr(out))
    return Ct(out, level, scale)


def mul_relin(ctx, keys, a, b):
    """Eq. 8 without rescale: tensor then relinearise; scale = product."""
    return relinearise(ctx, keys, tensor(ctx, a, b), a.level, a.scale * b.scale)


def _ks_rescale(ctx, d, ext, level, key):
    """Key inner product of d2's ModUp, then (d0, d1) + KS(d2) divided by
    P q_level in one basis conversion (relinearise and rescale together)."""
    out = np.zeros((2, level, ctx.N), np.uint64)
    ctx.L_.or_relin_rescale(ctx.h, ptr(np.ascontiguousarray(d[:2])), ptr(ext), level, ptr(key),
                            ptr(out))
    return out


def relin_rescale(ctx, keys, d, level, scale):
    """(d0, d1, d2) at `level` -> relinearised and rescaled to level - 1."""
    if level < 1:
        raise ValueError("level exhausted")
    ext = _modup(ctx, d[2], level)
    out = _ks_rescale(ctx, d, ext, level, keys.relin)
    s = scale / ctx.q[level]
    dl = ctx.delta[level - 1]
    if abs(s / dl - 1.0) < SNAP:
        s = dl
    return Ct(out, level - 1, s)


def mul(ctx, keys, a, b):
    """Eq. 8: align both to the lower level, multiply, relinearise and
    rescale (one division by P q_level)."""
    lv = min(a.level, b.level)
    a = level_down(ctx, a, lv)
    b = level_down(ctx, b, lv)
    return relin_rescale(ctx, keys, tensor(ctx, a, b), lv, a.scale * b.scale)


def mul_sum(ctx, keys, pairs):
    """sum_k a_k (x) b_k with a single relinearisation and rescale."""
    lv = min(min(a.level, b.level) for a, b in pairs)
    acc = None
    scale = None
    for a, b in pairs:
        a = level_down(ctx, a, lv)
        b = level_down(ctx, b, lv)
        d = tensor(ctx, a, b)
        if acc is None:
            acc, scale = d, a.scale * b.scale
        else:
            o = np.zeros_like(acc)
            ctx.L_.or_add(ctx.h, ptr(acc), ptr(d), 3, lv + 1, 0, ptr(o))
            acc = o
    return relin_rescale(ctx, keys, acc, lv, scale)


def rotate_many(ctx, keys, a, steps):
    """Eq. 10 for several steps sharing one ModUp (hoisted rotations).

    The automorphism X -> X^g is applied to the ModUp output (canonical
    form), so a single rotation and a hoisted one agree bit for bit.
    """
    out = {}
    ext = None
    for t in steps:
        g = ctx.galois(t)
        if g == 1:
            out[t] = a.copy()
            continue
        if ext is None:
            ext = _modup(ctx, a.data[1], a.level)
        if g not in keys.galois:
            raise KeyError("missing Galois key for step %d" % t)
        o = _ks(ctx, ext, a.level, keys.galois[g], g)
        c0 = np.zeros((a.level + 1, ctx.N), np.uint64)
        ctx.L_.or_automorphism_polys(ctx.h, ptr(np.ascontiguousarray(a.data[0])), a.level + 1, g, ptr(c0))
        res = np.zeros_like(a.data)
        ctx.L_.or_add(ctx.h, ptr(c0), ptr(o[0]), 1, a.level + 1, 0, ptr(res[0]))
        res[1] = o[1]
        out[t] = Ct(res, a.level, a.scale)
    return out


def rotate(ctx, keys, a, step):
    return rotate_many(ctx, keys, a, [step])[step]


# ---------------------------------------------------------------- double hoisting
# The baby steps of a BSGS matrix-vector product can stay in the extended
# basis QP_l (Bossuat et al. 2021, "double hoisting"; a reading of the BSGS
# matvec's hoisted rotations): each rotation skips its ModDown, the diagonal
# products and their sum are taken over QP_l, and the sum is divided by
# P q_level once per giant step (the rescale of the diagonal products and the
# ModDown of the rotations in one rounded division).
def _qp_rows(ctx, level):
    return list(range(level + 1)) + [ctx.L + 1 + k for k in range(ctx.alpha)]


def encode_qp(ctx, v, level, scale):
    """Plaintext of v over QP_level: [l + alpha][N] NTT form, the encoding's
    integer coefficients reduced mod each Q limb and special prime (the Q
    rows equal encode()'s)."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    co = np.zeros(ctx.N, np.int64)
    if ctx.L_.or_encode(ptr(v), len(v), ctx.log_n, scale, ptr(co)) != 0:
        raise OverflowError("oracle: encoding overflow")
    rows = _qp_rows(ctx, level)
    out = np.zeros((len(rows), ctx.N), np.uint64)
    for r, t in enumerate(rows):
        out[r] = np.mod(co, np.int64(ctx.moduli[t])).astype(np.uint64)
        ctx.L_.or_ntt_limb(ctx.h, ptr(out[r]), t, 0)
    return out


def rotate_many_qp(ctx, keys, a, steps):
    """Rotations of `a` kept in QP_l (no ModDown): {t: [2][l + alpha][N]}
    with R_t = (P sigma_t(c0) + acc_0, acc_1), acc the key inner product of
    sigma_t(ModUp(c1)); R_t decrypts to P rot(a, t) under the secret over
    QP_l. t = 0 (identity) gives (P c0, P c1)."""
    lv, rows = a.level, a.level + 1 + ctx.alpha
    out, ext = {}, None
    for t in steps:
        g = ctx.galois(t)
        R = np.zeros((2, rows, ctx.N), np.uint64)
        if g == 1:
            for k in range(2):
                ctx.L_.or_qp_lift(ctx.h, ptr(np.ascontiguousarray(a.data[k])), lv, 0, None, ptr(R[k]))
        else:
            if ext is None:
                ext = _modup(ctx, a.data[1], lv)
            if g not in keys.galois:
                raise KeyError("missing Galois key for step %d" % t)
            acc = np.zeros((2, rows, ctx.N), np.uint64)
            ctx.L_.or_key_product(ctx.h, ptr(ext), lv, ptr(keys.galois[g]), g, ptr(acc))
            ctx.L_.or_qp_lift(ctx.h, ptr(np.ascontiguousarray(a.data[0])), lv, g, ptr(acc[0]), ptr(R[0]))
            R[1] = acc[1]
        out[t] = R
    return out


def qp_mul_plain_acc(ctx, R, pt, level, acc):
    """acc += R * pt over QP_level (in place)."""
    ctx.L_.or_qp_mul_plain_acc(ctx.h, ptr(R), ptr(pt), level, ptr(acc))


def div_p_ql(ctx, acc, level, scale):
    """The QP_level pair acc ([2][l + alpha][N]) divided by P q_level with
    rounding to nearest (centred conversion of the dropped limbs): a
    ciphertext at level - 1 with scale `scale` / q_level (snapped to the
    canonical scale within 2^-30)."""
    if level < 1:
        raise ValueError("level exhausted")
    out = np.zeros((2, level, ctx.N), np.uint64)
    ctx.L_.or_div_p_ql(ctx.h, None, ptr(np.ascontiguousarray(acc)), level, ptr(out))
    s = scale / ctx.q[level]
    d = ctx.delta[level - 1]
    if abs(s / d - 1.0) < SNAP:
        s = d
    return Ct(out, level - 1, s)
