"""CKKS bootstrapping on the oracle (test infrastructure only).

The paper's parameters bootstrap as in Lee et al. 2022 (Experiment Setup);
the configurations here are leveled, and this module is the oracle side of
bootstrapping, the "next" row after them. The pipeline (Cheon, Han, Kim,
Kim and Song 2018, with a polynomial for the modular reduction):

* ModRaise: a ciphertext at level 0 is read over the whole chain. Its
  coefficients decrypt to t = m + q0 I over the integers, I a small integer
  polynomial (|I| bounded by about half the secret's Hamming weight; a
  sparse secret keeps it small).
* CoeffToSlot: the slots z' = E t / Delta (E the decoding map from N real
  coefficients to N/2 complex slots) are turned into two ciphertexts whose
  real slots hold t_j / Delta for the lower and upper halves of the
  coefficients: [t_lo; t_hi] / Delta = G [z'; conj z'] with G the inverse of
  [[E_lo, E_hi], [conj E_lo, conj E_hi]], each block applied to z' and to
  its conjugate (the conjugation automorphism X -> X^-1) as a dense
  baby-step giant-step linear transform with complex diagonals; then a
  product by the exact constant 2^-e, 2^e >= (K + 1) c with c = q0 / Delta,
  gives y = t_j / (Delta 2^e) in [-1, 1]. The diagonals are applied 2^B
  larger (B = 12) and the constant is 2^-(e + B): the slots after ModRaise
  reach about 2^27 while y needs about 2^-40 absolute precision, which a
  diagonal of magnitude 2^-6 rounded at a 2^40 plaintext scale does not
  give. The constant 2^-(e + B) is applied as a 45-bit integer over two
  rescales (mul_const_wide): a one-level constant product would realise it
  as a 5-bit integer. (Folding 1 / ((K + 1) c) into the diagonals instead
  would leave their encodings about 11 bits.)
* EvalMod: the Chebyshev interpolant of g(y) = c / (2 pi) sin(2 pi 2^e y / c)
  on [-1, 1] (Paterson-Stockmeyer evaluation, the SiLU evaluator), since
  g(t / (Delta 2^e)) = c / (2 pi) sin(2 pi m / q0) = m / Delta up to a
  relative (2 pi m / q0)^2 / 6.
* SlotToCoeff: z = E_lo (m_lo / Delta) + E_hi (m_hi / Delta), two dense
  transforms with complex diagonals on the real-slot ciphertexts.

The dense transforms need N/2 diagonals each, so this form is for small
rings; a full-size ring takes the factored (FFT-like) transforms instead.
Every operation is an oracle operation (ciphertext arithmetic of ckks.py and
the C core), so a GPU schedule of the same steps can be checked word for
word against it.
"""
import math

import numpy as np

from . import ckks, kan_he
from ._lib import ptr


# ---------------------------------------------------------------- keys
def boot_steps(ctx):
    """Rotation steps of the dense transforms: baby steps 1 .. g1 - 1 and
    giant steps g1 i over the N/2 slots."""
    n = ctx.slots
    g1 = 1 << ((n.bit_length() - 1 + 1) // 2)
    return list(range(1, g1)) + [g1 * i for i in range(1, n // g1)]


class BootKeys:
    """The secret (dense ternary, or sparse of Hamming weight h, which keeps
    the ModRaise overflow small), the relinearisation key, the transforms'
    rotation keys and the conjugation key (Galois element 2N - 1)."""

    _switch_key = ckks.Keys._switch_key

    def __init__(self, ctx, seed, h=None):
        self.ctx, self.seed, self.h = ctx, seed, h
        self.s = np.zeros((ctx.n_qp, ctx.N), np.uint64)
        self.s_coef = np.zeros(ctx.N, np.int64)
        if h is None:
            ctx.L_.or_keygen_secret(ctx.h, seed, ptr(self.s), ptr(self.s_coef))
        else:
            ctx.L_.or_keygen_secret_sparse(ctx.h, seed, int(h), ptr(self.s), ptr(self.s_coef))
        self.relin = self._switch_key(0)
        self.galois = {}
        for g in [ctx.galois(t) for t in boot_steps(ctx)] + [2 * ctx.N - 1]:
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


def linear_transform(ctx, keys, v, U):
    """Slots z -> U z (U: N/2 x N/2 complex) by baby-step giant-step over the
    N/2 cyclic diagonals u_t[s] = U[s][(s + t) mod n], hoisted baby steps;
    the diagonal products are accumulated and rescaled once per giant step
    (one level)."""
    n = ctx.slots
    g1 = 1 << ((n.bit_length() - 1 + 1) // 2)
    g2 = n // g1
    s = np.arange(n)
    baby = ckks.rotate_many(ctx, keys, v, list(range(g1)))
    lv = v.level
    Spt = ckks.plain_scale(ctx, v.scale, lv)
    z = None
    for i in range(g2):
        acc = None
        for j in range(g1):
            t = g1 * i + j
            d = U[s, (s + t) % n]
            d = np.roll(d, g1 * i)  # rot(d, -g1 i)
            pt = encode_complex(ctx, d, lv, Spt)
            prod = np.zeros_like(v.data)
            ctx.L_.or_mul_plain(ctx.h, ptr(baby[j].data), ptr(pt), 2, lv + 1, ptr(prod))
            if acc is None:
                acc = prod
            else:
                o = np.zeros_like(acc)
                ctx.L_.or_add(ctx.h, ptr(acc), ptr(prod), 2, lv + 1, 0, ptr(o))
                acc = o
        inner = ckks.rescale(ctx, ckks.Ct(acc, lv, v.scale * Spt))
        if i > 0:
            inner = ckks.rotate(ctx, keys, inner, g1 * i)
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


def coeff_to_slot_matrices(ctx):
    """(A_lo, B_lo, A_hi, B_hi): t_lo / Delta = A_lo z' + B_lo conj(z'), t_hi
    likewise."""
    n = ctx.slots
    E = decode_matrix(ctx)
    El, Eh = E[:, :n], E[:, n:]
    big = np.block([[El, Eh], [El.conj(), Eh.conj()]])
    Gm = np.linalg.inv(big)
    return Gm[:n, :n], Gm[:n, n:], Gm[n:, :n], Gm[n:, n:]


def mod_exponent(ctx, K):
    """e with 2^e >= (K + 1) q0 / Delta_0: y = t / (Delta 2^e) stays in [-1, 1]."""
    return math.ceil(math.log2((K + 1) * ctx.q[0] / ctx.delta[0]))


DIAG_BOOST = 12  # bits by which the CoeffToSlot diagonals are applied larger


def mul_const_wide(ctx, a, c):
    """a * c for a constant far below 1: mul_const realises c as
    rint(c S) / S with S near Delta, a relative error of 1 / (2 c S) (for
    c = 2^-35 about 1 %); here c is realised as an integer of about 45 bits,
    rint(c S2) with S2 = Delta_(l-2) q_l q_(l-1) / scale, and the product is
    rescaled twice, landing on the canonical scale of level l - 2 (two
    levels)."""
    lv = a.level
    S2 = ctx.delta[lv - 2] * float(ctx.q[lv]) * float(ctx.q[lv - 1]) / a.scale
    k = ckks.round_const(c, S2)
    once = ckks.rescale(ctx, ckks.Ct(ckks.mul_int(ctx, a, k).data, lv, a.scale * S2))
    return ckks.rescale(ctx, once)


def coeff_to_slot(ctx, keys, ct, K):
    A_lo, B_lo, A_hi, B_hi = (M * 2.0 ** DIAG_BOOST for M in coeff_to_slot_matrices(ctx))
    cj = conjugate(ctx, keys, ct)
    lo = ckks.add(ctx, linear_transform(ctx, keys, ct, A_lo), linear_transform(ctx, keys, cj, B_lo))
    hi = ckks.add(ctx, linear_transform(ctx, keys, ct, A_hi), linear_transform(ctx, keys, cj, B_hi))
    f = 2.0 ** -(mod_exponent(ctx, K) + DIAG_BOOST)
    return mul_const_wide(ctx, lo, f), mul_const_wide(ctx, hi, f)


def eval_mod_coeffs(ctx, K, degree):
    """Chebyshev coefficients (basis of [-1, 1]) of the interpolant of
    g(y) = c / (2 pi) sin(2 pi 2^e y / c) at the degree + 1 Chebyshev points."""
    c = ctx.q[0] / ctx.delta[0]
    w = 2.0 * math.pi * 2.0 ** mod_exponent(ctx, K) / c
    g = lambda y: c / (2.0 * math.pi) * np.sin(w * y)
    return np.polynomial.chebyshev.chebinterpolate(g, degree)


def eval_mod(ctx, keys, ct, K, degree):
    return kan_he.eval_cheb(ctx, keys, ct, eval_mod_coeffs(ctx, K, degree))


def slot_to_coeff(ctx, keys, lo, hi):
    n = ctx.slots
    E = decode_matrix(ctx)
    lv = min(lo.level, hi.level)
    lo, hi = ckks.level_down(ctx, lo, lv), ckks.level_down(ctx, hi, lv)
    return ckks.add(ctx, linear_transform(ctx, keys, lo, E[:, :n]),
                    linear_transform(ctx, keys, hi, E[:, n:]))


def bootstrap(ctx, keys, ct, K, degree):
    """A level-0 ciphertext back at a high level with the same slots (up to
    the precision the modular-reduction polynomial and the noise allow)."""
    raised = mod_raise(ctx, ct)
    lo, hi = coeff_to_slot(ctx, keys, raised, K)
    lo, hi = eval_mod(ctx, keys, lo, K, degree), eval_mod(ctx, keys, hi, K, degree)
    return slot_to_coeff(ctx, keys, lo, hi)
