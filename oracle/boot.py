"""CKKS bootstrapping on the oracle (test infrastructure only).

The paper's parameters bootstrap as in Lee et al. 2022 (Experiment Setup);
the configurations here are leveled, and this module is the oracle side of
bootstrapping, the "next" row after them. The pipeline (Cheon, Han, Kim,
Kim and Song 2018, with a polynomial for the modular reduction):

* ModRaise: a ciphertext at level 0 is read over the whole chain. Its
  coefficients decrypt to t = m + q0 I over the integers, I a small integer
  polynomial (|I| bounded by about half the secret's Hamming weight; a
  sparse secret keeps it small).
* CoeffToSlot: the slots are z = U w with w = (t_lo + i t_hi) / Delta (the
  n = N/2 complex coefficients, U the encoder's decoding map). U factors
  into log2(n) radix-2 stages and a bit reversal (the "special FFT"); the
  stages' inverses, merged a few at a time into levels of 2^(r+1) - 1
  cyclic diagonals each and applied by baby-step giant-step with hoisted
  baby rotations, give n BR(w) (the bit-reversed order is kept: EvalMod is
  slot-wise and SlotToCoeff undoes it). The conjugation automorphism
  X -> X^-1 splits real and imaginary parts (the latter times -i, the
  monomial X^(3N/2)); the exact constant 2^-(e + log2(2n)), applied as a
  wide integer over two rescales (mul_const_wide), gives
  y = t_j / (Delta 2^e) in [-1, 1] with 2^e >= (K + 1) c, c = q0 / Delta.
  The diagonals keep magnitude 1 (the inverse stages' halvings go into the
  final constant), so their encodings keep the plaintext scale's precision.
* EvalMod: the Chebyshev interpolant of g(y) = c / (2 pi) sin(2 pi 2^e y / c)
  on [-1, 1] (Paterson-Stockmeyer evaluation, the SiLU evaluator), since
  g(t / (Delta 2^e)) = c / (2 pi) sin(2 pi m / q0) = m / Delta up to a
  relative (2 pi m / q0)^2 / 6.
* SlotToCoeff: the two real halves joined as m_lo + i m_hi (i = X^(N/2)),
  then the merged forward stages: U (m / Delta), the original slots.

Precision follows q0 / Delta: EvalMod multiplies the absolute noise of y
(about 2^-30 at 40-bit scale primes) by 2^e, about (K + 1) q0 / Delta. Every
operation is an oracle operation (ciphertext arithmetic of ckks.py and the
C core), so a GPU schedule of the same steps can be checked word for word
against it.
"""
import math

import numpy as np

from . import ckks, kan_he
from ._lib import ptr


# ---------------------------------------------------------------- keys
class BootKeys:
    """The secret (dense ternary, or sparse of Hamming weight h, which keeps
    the ModRaise overflow small), the relinearisation key, rotation keys for
    `steps` and the conjugation key (Galois element 2N - 1)."""

    _switch_key = ckks.Keys._switch_key

    def __init__(self, ctx, seed, steps=(), h=None):
        self.ctx, self.seed, self.h = ctx, seed, h
        self.s = np.zeros((ctx.n_qp, ctx.N), np.uint64)
        self.s_coef = np.zeros(ctx.N, np.int64)
        if h is None:
            ctx.L_.or_keygen_secret(ctx.h, seed, ptr(self.s), ptr(self.s_coef))
        else:
            ctx.L_.or_keygen_secret_sparse(ctx.h, seed, int(h), ptr(self.s), ptr(self.s_coef))
        self.relin = self._switch_key(0)
        self.galois = {}
        for g in [ctx.galois(t) for t in steps] + [2 * ctx.N - 1]:
            if g != 1 and g not in self.galois:
                self.galois[g] = self._switch_key(g)


# ---------------------------------------------------------------- helpers
def decode_matrix(ctx):
    """E (N/2 x N complex): slots of the coefficient vector e_i in column i
    (the decoding map of the encoder, coefficient values in value units)."""
    N, n = ctx.N, ctx.slots
    E = np.zeros((n, N), complex)
    re, im = np.zeros(n), np.zeros(n)
    for i in range(N):
        m = np.zeros(N)
        m[i] = 1.0
        ctx.L_.or_decode_complex(ptr(m), ctx.log_n, ptr(re), ptr(im), n)
        E[:, i] = re + 1j * im
    return E


def decrypt_coeffs_crt(ctx, keys, ct):
    """Coefficients of c0 + c1 s over all of ct's limbs as centred Python
    integers (CRT of the limbs to Z / Q_l), so values beyond q0 / 2 come out
    whole (small rings only)."""
    l, N = ct.level + 1, ctx.N
    xs = []
    for t in range(l):
        q = int(ctx.q[t])
        v = (ct.data[0, t].astype(object) + ct.data[1, t].astype(object) * keys.s[t].astype(object)) % q
        a = np.array([int(u) for u in v], dtype=np.uint64)
        ctx.L_.or_ntt_limb(ctx.h, ptr(a), t, 1)
        xs.append(a)
    Q = 1
    for t in range(l):
        Q *= int(ctx.q[t])
    out = []
    for i in range(N):
        x = 0
        for t in range(l):
            qt = int(ctx.q[t])
            Qt = Q // qt
            x += int(xs[t][i]) * Qt * pow(Qt, -1, qt)
        x %= Q
        out.append(x - Q if 2 * x > Q else x)
    return out


def decode_complex(ctx, coeffs):
    """Complex slots of real coefficients given in value units."""
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    re, im = np.zeros(ctx.slots), np.zeros(ctx.slots)
    ctx.L_.or_decode_complex(ptr(c), ctx.log_n, ptr(re), ptr(im), ctx.slots)
    return re + 1j * im


def decrypt_crt(ctx, keys, ct):
    """Complex slots of ct decrypted over all its limbs."""
    return decode_complex(ctx, [x / ct.scale for x in decrypt_coeffs_crt(ctx, keys, ct)])


def conjugate(ctx, keys, a):
    """X -> X^(2N-1): the slots' complex conjugates (hoisted-rotation form)."""
    g = 2 * ctx.N - 1
    ext = ckks._modup(ctx, a.data[1], a.level)
    o = ckks._ks(ctx, ext, a.level, keys.galois[g], g)
    c0 = np.zeros((a.level + 1, ctx.N), np.uint64)
    ctx.L_.or_automorphism_polys(ctx.h, ptr(np.ascontiguousarray(a.data[0])), a.level + 1, g, ptr(c0))
    res = np.zeros_like(a.data)
    ctx.L_.or_add(ctx.h, ptr(c0), ptr(o[0]), 1, a.level + 1, 0, ptr(res[0]))
    res[1] = o[1]
    return ckks.Ct(res, a.level, a.scale)


def encode_complex(ctx, z, level, scale):
    z = np.asarray(z, complex)
    re, im = np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)
    pt = np.zeros((level + 1, ctx.N), np.uint64)
    if ctx.L_.or_encode_plain_complex(ctx.h, ptr(re), ptr(im), len(z), level, scale, ptr(pt)) != 0:
        raise OverflowError("oracle: encoding overflow")
    return pt


def mul_monomial(ctx, a, k):
    """a X^k (exact, no level): every slot times zeta_j^k; X^(N/2)
    multiplies every slot by i, since zeta_j^(N/2) = i^(5^j) = i."""
    k %= 2 * ctx.N
    l = a.level + 1
    pt = np.zeros((l, ctx.N), np.uint64)
    for t in range(l):
        if k < ctx.N:
            pt[t, k] = 1
        else:
            pt[t, k - ctx.N] = ctx.q[t] - 1
        ctx.L_.or_ntt_limb(ctx.h, ptr(pt[t]), t, 0)
    out = np.zeros_like(a.data)
    ctx.L_.or_mul_plain(ctx.h, ptr(np.ascontiguousarray(a.data)), ptr(pt), 2, l, ptr(out))
    return ckks.Ct(out, a.level, a.scale)


# ---------------------------------------------------------------- the slot transforms
# Slot j of the encoder holds sum_i w_i zeta_j^i over the n = N/2 complex
# coefficients w_i = m_i + i m_(i+n), zeta_j = zeta^(5^j mod 2N): z = U w.
# U factors as F_(log n) ... F_1 BR (decimation in time, BR the bit
# reversal): stage s pairs slots p and p + h (h = 2^(s-1), blocks of 2h) as
#   out[p] = x[p] + w_r x[p + h],  out[p + h] = x[p] - w_r x[p + h],
# r = p mod 2h < h, w_r = exp(2 pi i (5^r mod 8h) / (8h)) (the root of the
# half-size problem on 2h slots). As cyclic diagonals of the slot vector
# (offset o: the factor of rot(x, o), rot moving slot p + o to p) a stage has
# offsets 0, +h, -h; r stages merged have offsets k 2^a, |k| < 2^r.
ROOT_LOG = 17  # every stage root is a 2^17-th root of unity (N <= 2^16)


def _cos_sin_decimal(k, log_m):
    """(cos, sin)(2 pi k / 2^log_m) for 0 <= k <= 2^log_m / 8, correctly
    rounded to double from a 40-digit Taylor series (the same bits on every
    machine, unlike a platform math library)."""
    from decimal import Decimal, getcontext
    getcontext().prec = 40
    pi = Decimal("3.141592653589793238462643383279502884197169399375")
    x = 2 * pi * k / (Decimal(2) ** log_m)
    c = s = Decimal(0)
    term = Decimal(1)  # x^n / n!
    for n in range(0, 60):
        if n % 4 == 0:
            c += term
        elif n % 4 == 1:
            s += term
        elif n % 4 == 2:
            c -= term
        else:
            s -= term
        term = term * x / (n + 1)
    return float(c), float(s)


_ROOTS = {}


def _root_table(log_m):
    """(cos, sin)(2 pi k / 2^log_m) for every k, from the first octant by the
    exact symmetries cos(pi/2 - t) = sin t and quarter turns."""
    if log_m in _ROOTS:
        return _ROOTS[log_m]
    M = 1 << log_m
    o = M // 8
    base = [_cos_sin_decimal(k, log_m) for k in range(o + 1)]
    cs = np.zeros(M)
    sn = np.zeros(M)
    for k in range(M // 4 + 1):  # first quadrant
        if k <= o:
            c, s_ = base[k]
        else:
            s_, c = base[M // 4 - k]
        cs[k % M], sn[k % M] = c, s_
    for k in range(M // 4 + 1, M):
        q, r = divmod(k, M // 4)
        c, s_ = cs[r], sn[r]
        for _ in range(q):  # times i: (c, s) -> (-s, c)
            c, s_ = -s_, c
        cs[k], sn[k] = c, s_
    _ROOTS[log_m] = (cs, sn)
    return _ROOTS[log_m]


def _stage_roots(h):
    """w_r = exp(2 pi i (5^r mod 8h) / (8h)) for r < h: the 2^17-th roots
    of unity at k = (5^r mod 8h) 2^17 / (8h)."""
    cs, sn = _root_table(ROOT_LOG)
    k = np.array([pow(5, int(x), 8 * h) for x in range(h)], dtype=np.int64) * ((1 << ROOT_LOG) // (8 * h))
    return cs[k] + 1j * sn[k]


def _cmul(a, b):
    """a * b elementwise with each real product and sum rounded once (the
    same bits on every machine)."""
    re = np.subtract(np.multiply(a.real, b.real), np.multiply(a.imag, b.imag))
    im = np.add(np.multiply(a.real, b.imag), np.multiply(a.imag, b.real))
    return re + 1j * im


def fft_stage(ctx, s, inverse=False):
    """{offset: diagonal} of F_s, or of 2 F_s^-1 (inverse): from the pair
    (u + w v, u - w v) the inverse recovers (2u, 2 conj(w) v)."""
    n = ctx.slots
    h = 1 << (s - 1)
    p = np.arange(n)
    r = p % (2 * h)
    lower = r < h
    w = _stage_roots(h)[np.where(lower, r, r - h)]
    one, zero = np.ones(n, complex), np.zeros(n, complex)
    if not inverse:
        terms = [(0, np.where(lower, one, -w)), (h, np.where(lower, w, zero)),
                 (-h, np.where(lower, zero, one))]
    else:
        terms = [(0, np.where(lower, one, -w.conj())), (h, np.where(lower, one, zero)),
                 (-h, np.where(lower, zero, w.conj()))]
    d = {}
    for o, v in terms:  # offsets mod n: at h = n/2, +h and -h are one rotation
        d[o % n] = d[o % n] + v if o % n in d else v
    return d


def compose(ctx, A, B):
    """Diagonals of the product A B (B applied first):
    (A B)_o = sum over a + b = o (mod n) of A_a (.) rot(B_b, a)."""
    n = ctx.slots
    out = {}
    for a in sorted(A):
        for b in sorted(B):
            o = (a + b) % n
            term = _cmul(A[a], np.roll(B[b], -a))
            out[o] = out[o] + term if o in out else term
    return out


def _groups(n_stages, n_levels, ascending):
    sizes = [n_stages // n_levels + (1 if i < n_stages % n_levels else 0) for i in range(n_levels)]
    stages = list(range(1, n_stages + 1)) if ascending else list(range(n_stages, 0, -1))
    out, k = [], 0
    for sz in sizes:
        out.append(stages[k:k + sz])
        k += sz
    return out


class LinearTransform:
    """z -> sum_k d_k (.) rot(z, base + k stride), k in [0, len(diags)), by
    baby-step giant-step: baby steps j stride (j < g1, one hoisted ModUp),
    giant steps base + g1 i stride; an all-zero diagonal is skipped. form
    "single": hoisted baby rotations, one rescale per giant step; "double":
    the baby rotations kept in QP_l and each giant step's products divided by
    P q_l once (double hoisting)."""

    def __init__(self, base, stride, diags, g1=None, form="single"):
        if form not in ("single", "double"):
            raise ValueError(form)
        self.base, self.stride, self.form = int(base), int(stride), form
        self.diags = [np.asarray(d, complex) for d in diags]
        K = len(self.diags)
        self.g1 = g1 or 1 << max(0, math.ceil(math.log2(math.sqrt(K))))
        self.g2 = -(-K // self.g1)

    def matrix_apply(self, z):
        """The transform on plain slots (numpy)."""
        return sum(d * np.roll(z, -(self.base + k * self.stride)) for k, d in enumerate(self.diags))

    def steps(self, n):
        st = {(j * self.stride) % n for j in range(1, self.g1)}
        st |= {(self.base + self.g1 * i * self.stride) % n for i in range(self.g2)}
        return sorted(st - {0})


def transform_levels(ctx, n_levels, inverse, form="single"):
    """The merged levels of U's factors: SlotToCoeff (inverse False) applies
    F_1 .. F_(log n) in that order, CoeffToSlot (inverse True) applies
    2 F_(log n)^-1 .. 2 F_1^-1. Each level merges consecutive stages with
    h = 2^a .. 2^(a+r-1): offsets k 2^a, k from -(2^r - 1) to 2^r - 1."""
    n = ctx.slots
    log_n = n.bit_length() - 1
    out = []
    for grp in _groups(log_n, n_levels, ascending=not inverse):
        M = None
        for s in grp:
            st = fft_stage(ctx, s, inverse)
            M = st if M is None else compose(ctx, st, M)
        a, r = min(grp) - 1, len(grp)
        stride, span = 1 << a, (1 << r) - 1
        base = -span * stride
        diags, seen = [], set()
        for k in range(2 * span + 1):
            o = (base + k * stride) % n
            if o in M and o not in seen:
                diags.append(M[o])
                seen.add(o)
            else:
                diags.append(np.zeros(n, complex))
        out.append(LinearTransform(base, stride, diags, form=form))
    return out


def encode_qp_complex(ctx, z, level, scale):
    """Plaintext of the complex slots z over QP_level ([l + alpha][N], NTT
    form): the encoding's integer coefficients reduced mod each Q limb and
    special prime (the Q rows equal encode_complex's)."""
    z = np.asarray(z, complex)
    re, im = np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)
    co = np.zeros(ctx.N, np.int64)
    if ctx.L_.or_encode_complex(ptr(re), ptr(im), len(z), ctx.log_n, scale, ptr(co)) != 0:
        raise OverflowError("oracle: encoding overflow")
    rows = list(range(level + 1)) + [ctx.L + 1 + k for k in range(ctx.alpha)]
    out = np.zeros((len(rows), ctx.N), np.uint64)
    for r, t in enumerate(rows):
        out[r] = np.mod(co, np.int64(ctx.moduli[t])).astype(np.uint64)
        ctx.L_.or_ntt_limb(ctx.h, ptr(out[r]), t, 0)
    return out


def linear_transform(ctx, keys, v, lt):
    """The BSGS evaluation of a LinearTransform: per giant step i the
    products of the baby rotations with the diagonals pre-rotated by
    -(base + g1 i stride), summed, rescaled once (one level), then rotated
    by base + g1 i stride. In the double form the baby rotations stay in
    QP_l, the products and sum are taken over QP_l and the rescale is the
    division of the sum by P q_l."""
    if lt.form == "double":
        return _linear_transform_double(ctx, keys, v, lt)
    n = ctx.slots
    baby = ckks.rotate_many(ctx, keys, v, [j * lt.stride for j in range(lt.g1)])
    lv = v.level
    Spt = ckks.plain_scale(ctx, v.scale, lv)
    z = None
    for i in range(lt.g2):
        G = lt.base + lt.g1 * i * lt.stride
        acc = None
        for j in range(lt.g1):
            k = lt.g1 * i + j
            if k >= len(lt.diags) or not lt.diags[k].any():
                continue
            pt = encode_complex(ctx, np.roll(lt.diags[k], G), lv, Spt)
            prod = np.zeros_like(v.data)
            ctx.L_.or_mul_plain(ctx.h, ptr(baby[j * lt.stride].data), ptr(pt), 2, lv + 1, ptr(prod))
            if acc is None:
                acc = prod
            else:
                o = np.zeros_like(acc)
                ctx.L_.or_add(ctx.h, ptr(acc), ptr(prod), 2, lv + 1, 0, ptr(o))
                acc = o
        if acc is None:
            continue
        inner = ckks.rescale(ctx, ckks.Ct(acc, lv, v.scale * Spt))
        if G % n:
            inner = ckks.rotate(ctx, keys, inner, G % n)
        z = inner if z is None else ckks.add(ctx, z, inner)
    return z


def _linear_transform_double(ctx, keys, v, lt):
    n = ctx.slots
    R = ckks.rotate_many_qp(ctx, keys, v, [j * lt.stride for j in range(lt.g1)])
    lv = v.level
    Spt = ckks.plain_scale(ctx, v.scale, lv)
    z = None
    for i in range(lt.g2):
        G = lt.base + lt.g1 * i * lt.stride
        acc, any_ = np.zeros_like(R[0]), False
        for j in range(lt.g1):
            k = lt.g1 * i + j
            if k >= len(lt.diags) or not lt.diags[k].any():
                continue
            pt = encode_qp_complex(ctx, np.roll(lt.diags[k], G), lv, Spt)
            ckks.qp_mul_plain_acc(ctx, R[j * lt.stride], pt, lv, acc)
            any_ = True
        if not any_:
            continue
        inner = ckks.div_p_ql(ctx, acc, lv, v.scale * Spt)
        if G % n:
            inner = ckks.rotate(ctx, keys, inner, G % n)
        z = inner if z is None else ckks.add(ctx, z, inner)
    return z


# ---------------------------------------------------------------- the pipeline
def mod_raise(ctx, ct, level=None):
    if ct.level != 0:
        raise ValueError("ModRaise takes a level-0 ciphertext")
    level = ctx.L if level is None else level
    out = np.zeros((2, level + 1, ctx.N), np.uint64)
    ctx.L_.or_mod_raise(ctx.h, ptr(np.ascontiguousarray(ct.data)), level, ptr(out))
    return ckks.Ct(out, level, ct.scale)


def mod_exponent(ctx, K):
    """e with 2^e >= (K + 1) q0 / Delta_0: y = t / (Delta 2^e) stays in [-1, 1]."""
    return math.ceil(math.log2((K + 1) * ctx.q[0] / ctx.delta[0]))


def mul_bigint(ctx, a, k):
    """a times the integer k of any size: limb t times k mod q_t (the
    constant polynomial's transform is k in every position)."""
    l = a.level + 1
    pt = np.zeros((l, ctx.N), np.uint64)
    for t in range(l):
        pt[t, :] = k % ctx.q[t]
    out = np.zeros_like(a.data)
    ctx.L_.or_mul_plain(ctx.h, ptr(np.ascontiguousarray(a.data)), ptr(pt), 2, l, ptr(out))
    return ckks.Ct(out, a.level, a.scale)


def mul_const_wide(ctx, a, c):
    """a * c for a constant far below 1, landing on the canonical scale of
    level l - 2 (two levels). A one-level constant product realises c as
    rint(c S) / S with S near the prime size, a relative error 1 / (2 c S)
    that EvalMod would multiply by about c K q0 / Delta; here c is realised
    as the integer k = rint(c S2), S2 = Delta_(l-2) q_l q_(l-1) / scale
    (rounded in double precision, a relative error of 2^-53, the integer
    exact however large), and the product is rescaled twice."""
    lv = a.level
    S2 = ctx.delta[lv - 2] * float(ctx.q[lv]) * float(ctx.q[lv - 1]) / a.scale
    k = int(np.rint(c * S2))
    once = ckks.rescale(ctx, ckks.Ct(mul_bigint(ctx, a, k).data, lv, a.scale * S2))
    return ckks.rescale(ctx, once)


def coeff_to_slot(ctx, keys, ct, K, levels):
    """(y_lo, y_hi): real slots p holding t_(brv(p)) / (Delta 2^e) and
    t_(n + brv(p)) / (Delta 2^e) for the raised ciphertext's coefficients t.
    The merged levels of 2 F^-1 give n BR(w), w = (t_lo + i t_hi) / Delta;
    adding the conjugate gives 2 n Re, subtracting it and multiplying by
    -i = X^(3N/2) gives 2 n Im; the exact constant 2^-(e + log2(2n)) then
    brings both into [-1, 1] (two levels)."""
    for lt in levels:
        ct = linear_transform(ctx, keys, ct, lt)
    cj = conjugate(ctx, keys, ct)
    re2 = ckks.add(ctx, ct, cj)
    im2 = mul_monomial(ctx, ckks.sub(ctx, ct, cj), 3 * ctx.N // 2)
    f = 2.0 ** -(mod_exponent(ctx, K) + ctx.log_n)
    return mul_const_wide(ctx, re2, f), mul_const_wide(ctx, im2, f)


def eval_mod_coeffs(ctx, K, degree):
    """Chebyshev coefficients (basis of [-1, 1]) of the interpolant of
    g(y) = c / (2 pi) sin(2 pi 2^e y / c) at the degree + 1 Chebyshev points."""
    c = ctx.q[0] / ctx.delta[0]
    w = 2.0 * math.pi * 2.0 ** mod_exponent(ctx, K) / c
    g = lambda y: c / (2.0 * math.pi) * np.sin(w * y)
    return np.polynomial.chebyshev.chebinterpolate(g, degree)


def eval_mod(ctx, keys, ct, K, degree):
    return kan_he.eval_cheb(ctx, keys, ct, eval_mod_coeffs(ctx, K, degree))


def slot_to_coeff(ctx, keys, lo, hi, levels):
    """z = U (m_lo + i m_hi): the real-slot halves joined by X^(N/2) (times
    i), then the merged levels of F, which take the bit-reversed order the
    CoeffToSlot left back to the coefficients' order."""
    lv = min(lo.level, hi.level)
    lo, hi = ckks.level_down(ctx, lo, lv), ckks.level_down(ctx, hi, lv)
    ct = ckks.add(ctx, lo, mul_monomial(ctx, hi, ctx.N // 2))
    for lt in levels:
        ct = linear_transform(ctx, keys, ct, lt)
    return ct


class Plan:
    """The bootstrapping's fixed parts: the merged transform levels, the
    overflow bound K (|I| <= K) and the EvalMod polynomial's degree."""

    def __init__(self, ctx, K, degree, cts_levels=2, stc_levels=2, form="single"):
        self.K, self.degree = K, degree
        self.cts = transform_levels(ctx, cts_levels, inverse=True, form=form)
        self.stc = transform_levels(ctx, stc_levels, inverse=False, form=form)
        self.cheb = eval_mod_coeffs(ctx, K, degree)

    def steps(self, ctx):
        st = set()
        for lt in self.cts + self.stc:
            st |= set(lt.steps(ctx.slots))
        return sorted(st)


def bootstrap(ctx, keys, ct, plan):
    """A level-0 ciphertext back at a high level with the same slots (up to
    the precision the modular-reduction polynomial and the noise allow)."""
    raised = mod_raise(ctx, ct)
    lo, hi = coeff_to_slot(ctx, keys, raised, plan.K, plan.cts)
    lo = kan_he.eval_cheb(ctx, keys, lo, plan.cheb)
    hi = kan_he.eval_cheb(ctx, keys, hi, plan.cheb)
    return slot_to_coeff(ctx, keys, lo, hi, plan.stc)


def pack_tree(ctx, keys, cts, nb):
    """One ciphertext holding ciphertext b's slots [0, nb) at [b nb, b nb + nb)
    (the inputs already zero outside [0, nb)): pairs (c_2k, c_2k+1) become
    c_2k + rot(c_2k+1, -nb), then pairs of pairs with -2 nb, and so on."""
    cur, step = list(cts), nb
    while len(cur) > 1:
        nxt = []
        for k in range(0, len(cur), 2):
            if k + 1 < len(cur):
                nxt.append(ckks.add(ctx, cur[k], ckks.rotate(ctx, keys, cur[k + 1], -step)))
            else:
                nxt.append(cur[k])
        cur, step = nxt, step * 2
    return cur[0]


def unpack_tree(ctx, keys, packed, count, nb):
    """[rot(packed, b nb) for b < count], each by one rotation of an earlier
    one: u_(x + s) = rot(u_x, s nb) for s = top/2, top/4, .., 1."""
    out = {0: packed}
    s = 1 << max(0, (count - 1).bit_length() - 1) if count > 1 else 0
    while s >= 1:
        for x in sorted(out):
            if x + s < count and x + s not in out:
                out[x + s] = ckks.rotate(ctx, keys, out[x], s * nb)
        s //= 2
    return [out[b] for b in range(count)]


def refresh_packed(ctx, keys, hs, n_out, plan):
    """A batch refreshed with one bootstrap per S / nb ciphertexts (nb the
    least power of two >= n_out): each output masked to its slots [0, n_out)
    (one level), packed, brought to level 0, bootstrapped, unpacked."""
    nb = 1 << max(0, (n_out - 1).bit_length())
    per = ctx.slots // nb
    mask = np.ones(n_out)
    masked = [ckks.mul_plain(ctx, h, mask) for h in hs]
    out = []
    for g in range(0, len(masked), per):
        grp = masked[g:g + per]
        packed = pack_tree(ctx, keys, grp, nb)
        fresh = bootstrap(ctx, keys, ckks.level_down(ctx, packed, 0), plan)
        out.extend(unpack_tree(ctx, keys, fresh, len(grp), nb))
    return out


def infer_deep(ctx, keys, xs, model, plan, refresh_before, packed=False):
    """An encrypted KAN deeper than the chain, on the batch xs (a list of
    ciphertexts): before each layer index in refresh_before the batch is
    refreshed, each ciphertext brought to level 0 and bootstrapped, or, with
    packed, the whole batch through refresh_packed; the layers run as in
    kan_he.infer."""
    hs = list(xs)
    for i, layer in enumerate(model):
        if i in refresh_before:
            if packed:
                hs = refresh_packed(ctx, keys, hs, model[i - 1]["n_out"], plan)
            else:
                hs = [bootstrap(ctx, keys, ckks.level_down(ctx, h, 0), plan) for h in hs]
        hs = [kan_he.layer_eval(ctx, keys, h, layer) for h in hs]
    return hs
