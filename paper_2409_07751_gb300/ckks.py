"""ctypes binding of the C ABI in include/ckks_kan.h (argument marshalling only).

Every computation runs in `libckks_kan.so`; this module converts numpy
arrays to pointers and error codes to exceptions. Loading fails loudly if
the library has not been built.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libckks_kan.so")

_lib = None

c_u64, c_i64, c_i32, c_dbl, c_vp, c_sz = (ctypes.c_uint64, ctypes.c_int64, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t)
PP = ctypes.POINTER(ctypes.c_void_p)


class KanLayerDesc(ctypes.Structure):
    _fields_ = [("n_in", c_i32), ("n_out", c_i32), ("G", c_i32), ("k", c_i32),
                ("grid_lo", c_dbl), ("grid_hi", c_dbl),
                ("coef", c_vp), ("w_s", c_vp), ("w_b", c_vp),
                ("R", c_dbl), ("silu_lo", c_dbl), ("silu_hi", c_dbl),
                ("silu_cheb", c_vp), ("silu_degree", c_i32),
                ("comp", c_vp), ("n_comp", c_i32), ("naive", c_i32),
                ("comp_poly", c_vp), ("comp_poly_len", c_vp), ("n_comp_poly", c_i32),
                ("b0_form", c_i32), ("bsgs_form", c_i32)]


SIGNATURES = {
    "ckks_strerror": (ctypes.c_char_p, [c_i32]),
    "ckks_last_error": (ctypes.c_char_p, []),
    "ckks_context_create": (c_i32, [c_i32, c_i32, c_i32, c_i32, c_i32, c_i32, c_i32, PP]),
    "ckks_context_destroy": (c_i32, [c_vp]),
    "ckks_autotune_keyswitch": (c_i32, [c_i32, c_i32, c_i32, c_i32, c_i32, c_i32, c_i32, c_vp, c_vp,
                                        c_vp, c_vp, c_i32, c_vp]),
    "ckks_context_info": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "ckks_set_stream": (c_i32, [c_vp, c_vp]),
    "ckks_set_fusion": (c_i32, [c_vp, c_i32]),
    "ckks_synchronize": (c_i32, [c_vp]),
    "ckks_selftest_wait": (c_i32, [c_vp, c_i64]),
    "ckks_ntt": (c_i32, [c_vp, c_vp, c_sz, c_i32, c_i32]),
    "ckks_kernel_kind_count": (c_i32, []),
    "ckks_kernel_kind_name": (ctypes.c_char_p, [c_i32]),
    "ckks_launch_counts": (c_i32, [c_vp, c_vp, c_i32]),
    "ckks_profile_enable": (c_i32, [c_vp, c_i32]),
    "ckks_profile_collect": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i32]),
    "ckks_profile_collect2": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_i32]),
    "ckks_int_peak": (c_i32, [c_vp, c_i32, ctypes.POINTER(c_dbl)]),
    "ckks_autotune_ntt": (c_i32, [c_vp, c_i32, c_vp, c_vp]),
    "ckks_set_ntt_shape": (c_i32, [c_vp, c_i32, c_i32]),
    "ckks_keygen": (c_i32, [c_vp, c_u64, c_vp, c_sz, PP]),
    "ckks_keygen_ex": (c_i32, [c_vp, c_u64, c_i32, c_vp, c_sz, c_i32, c_u64, PP]),
    "ckks_keys_compress": (c_i32, [c_vp]),
    "ckks_keys_bytes": (c_i32, [c_vp, ctypes.POINTER(c_sz)]),
    "ckks_mod_raise": (c_i32, [c_vp, c_vp, c_i32, PP]),
    "ckks_conjugate": (c_i32, [c_vp, c_vp, c_vp, PP]),
    "ckks_mul_monomial": (c_i32, [c_vp, c_vp, c_i64, PP]),
    "ckks_mul_const_wide": (c_i32, [c_vp, c_vp, c_dbl, PP]),
    "ckks_lt_create": (c_i32, [c_vp, c_i32, c_dbl, c_i64, c_i64, c_sz, c_vp, c_vp, c_i32, c_i32,
                               PP]),
    "ckks_lt_destroy": (c_i32, [c_vp]),
    "ckks_lt_rotations": (c_i32, [c_vp, c_vp, c_sz, ctypes.POINTER(c_sz)]),
    "ckks_lt_apply": (c_i32, [c_vp, c_vp, c_vp, c_vp, PP]),
    "ckks_boot_create": (c_i32, [c_vp, c_i32, c_i32, c_i32, c_i32, c_i32, PP]),
    "ckks_boot_create_ex": (c_i32, [c_vp, c_i32, c_vp, c_sz, c_vp, c_sz, c_vp, c_sz, PP]),
    "ckks_boot_destroy": (c_i32, [c_vp]),
    "ckks_boot_info": (c_i32, [c_vp, ctypes.POINTER(c_i32), ctypes.POINTER(c_i32),
                               ctypes.POINTER(c_i32), ctypes.POINTER(c_sz)]),
    "ckks_boot_coefficients": (c_i32, [c_vp, c_vp, c_sz]),
    "ckks_boot_diagonals": (c_i32, [c_vp, c_i32, c_sz, ctypes.POINTER(c_i64),
                                    ctypes.POINTER(c_i64), ctypes.POINTER(c_sz)]),
    "ckks_boot_levels": (c_i32, [c_vp, c_i32, c_i32, c_sz, c_vp, c_vp, c_sz,
                                 ctypes.POINTER(c_i64), ctypes.POINTER(c_i64),
                                 ctypes.POINTER(c_sz)]),
    "ckks_boot_rotations": (c_i32, [c_vp, c_vp, c_sz, ctypes.POINTER(c_sz)]),
    "ckks_boot_coeff_to_slot": (c_i32, [c_vp, c_vp, c_vp, c_vp, PP, PP]),
    "ckks_boot_eval_mod": (c_i32, [c_vp, c_vp, c_vp, c_vp, PP]),
    "ckks_boot_slot_to_coeff": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, PP]),
    "ckks_bootstrap": (c_i32, [c_vp, c_vp, c_vp, c_vp, PP]),
    "kan_model_set_bootstrap": (c_i32, [c_vp, c_vp]),
    "kan_model_refresh_rotations": (c_i32, [c_vp, c_sz, c_vp, c_sz, ctypes.POINTER(c_sz)]),
    "ckks_keys_destroy": (c_i32, [c_vp]),
    "ckks_keys_export_secret": (c_i32, [c_vp, c_vp, c_sz]),
    "ckks_keys_export_switch": (c_i32, [c_vp, c_u64, c_vp, c_sz]),
    "ckks_galois_element": (c_u64, [c_vp, ctypes.c_int32]),
    "ckks_encrypt": (c_i32, [c_vp, c_vp, c_vp, c_sz, c_sz, c_i32, c_u64, c_u64, PP]),
    "ckks_decrypt": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_sz]),
    "ckks_ct_info": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "ckks_ct_export": (c_i32, [c_vp, c_vp, c_sz]),
    "ckks_ct_import": (c_i32, [c_vp, c_vp, c_sz, c_i32, c_dbl, PP]),
    "ckks_ct_import_async": (c_i32, [c_vp, c_vp, c_sz, c_i32, c_dbl, c_vp, PP]),
    "ckks_ct_slice": (c_i32, [c_vp, c_vp, c_sz, c_sz, PP]),
    "ckks_ct_destroy": (c_i32, [c_vp]),
    "ckks_add": (c_i32, [c_vp, c_vp, c_vp, PP]),
    "ckks_sub": (c_i32, [c_vp, c_vp, c_vp, PP]),
    "ckks_mul_relin": (c_i32, [c_vp, c_vp, c_vp, c_vp, PP]),
    "ckks_rescale": (c_i32, [c_vp, c_vp, PP]),
    "ckks_mul": (c_i32, [c_vp, c_vp, c_vp, c_vp, PP]),
    "ckks_rescale_noalloc": (c_i32, [c_vp, c_vp, c_sz, c_i32, c_vp]),
    "ckks_mul_plain": (c_i32, [c_vp, c_vp, c_vp, c_sz, PP]),
    "ckks_add_plain": (c_i32, [c_vp, c_vp, c_vp, c_sz, PP]),
    "ckks_mul_const": (c_i32, [c_vp, c_vp, c_dbl, PP]),
    "ckks_add_const": (c_i32, [c_vp, c_vp, c_dbl, PP]),
    "ckks_level_down": (c_i32, [c_vp, c_vp, c_i32, PP]),
    "ckks_rotate": (c_i32, [c_vp, c_vp, c_vp, ctypes.c_int32, PP]),
    "ckks_rotate_hoisted": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "kan_silu_fit": (c_i32, [c_dbl, c_dbl, c_dbl, c_dbl, c_i32, c_i32, c_i32, c_vp]),
    "kan_comp_minimax": (c_i32, [c_dbl, c_dbl, c_vp, c_i32, c_vp, c_vp]),
    "kan_calibrate": (c_i32, [c_vp, c_sz, c_vp, c_sz, c_i32, c_vp, c_i32, c_i32, c_vp, c_vp, c_vp,
                              c_vp]),
    "kan_model_create": (c_i32, [c_vp, c_vp, c_sz, PP]),
    "kan_model_destroy": (c_i32, [c_vp]),
    "kan_model_rotations": (c_i32, [c_vp, c_vp, c_sz, c_vp]),
    "kan_model_layer_depth": (c_i32, [c_vp, c_i32, c_vp]),
    "kan_model_layer_chunks": (c_i32, [c_vp, c_i32, c_vp, c_vp]),
    "kan_model_set_graphs": (c_i32, [c_vp, c_i32]),
    "kan_layer_eval": (c_i32, [c_vp, c_vp, c_vp, c_i32, c_vp, PP]),
    "kan_infer": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_sz, PP]),
    "kan_server_create": (c_i32, [c_vp, c_sz, PP]),
    "kan_server_destroy": (c_i32, [c_vp]),
    "kan_server_add_model": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "kan_server_submit": (c_i32, [c_vp, c_i32, c_vp, c_vp]),
    "kan_server_step": (c_i32, [c_vp, c_vp]),
    "kan_server_take": (c_i32, [c_vp, c_u64, PP]),
    "kan_server_status": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "kan_server_footprint": (c_i32, [c_vp, c_i32, c_vp]),
}

PENDING = 1


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libckks_kan.so is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class CkksError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (lib().ckks_strerror(code).decode(), code, msg))
        self.code = code


def check(rc):
    if rc != 0:
        raise CkksError(rc, lib().ckks_last_error().decode())


def _p(a):
    return a.ctypes.data if a is not None else None


def autotune_keyswitch(log_n, n_scale, max_qp_bits, batch=8, q0_bits=60, scale_bits=40, device=0):
    """(alpha, p_bits, {alpha: ms per HMult+HRot}) of the fastest digit layout."""
    a, p, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    tried = np.zeros(16, np.int32)
    ms = np.zeros(16)
    check(lib().ckks_autotune_keyswitch(log_n, q0_bits, scale_bits, n_scale, max_qp_bits, batch, device,
                                        ctypes.byref(a), ctypes.byref(p), _p(tried), _p(ms), 16,
                                        ctypes.byref(n)))
    return a.value, p.value, {int(t): float(m) for t, m in zip(tried[:n.value], ms[:n.value])}


class Context:
    def __init__(self, log_n, n_scale, n_special, q0_bits=60, scale_bits=40, p_bits=60, device=0):
        h = c_vp()
        check(lib().ckks_context_create(log_n, q0_bits, scale_bits, n_scale, p_bits, n_special,
                                        device, ctypes.byref(h)))
        self.h = h
        self.log_n, self.N, self.slots = log_n, 1 << log_n, 1 << (log_n - 1)
        self.L, self.alpha = n_scale, n_special
        n = ctypes.c_int()
        check(lib().ckks_context_info(h, None, None, ctypes.byref(n)))
        self.n_qp = n.value
        self.moduli = np.zeros(self.n_qp, np.uint64)
        self.delta = np.zeros(self.L + 1)
        check(lib().ckks_context_info(h, _p(self.moduli), _p(self.delta), None))
        self.beta_max = (self.L + 1 + self.alpha - 1) // self.alpha

    def close(self):
        if self.h:
            lib().ckks_context_destroy(self.h)
            self.h = None

    def synchronize(self):
        check(lib().ckks_synchronize(self.h))

    def selftest_wait(self, limit_cycles):
        """Runs one bounded device wait that cannot complete; returns the
        library's status code (CKKS_ERR_TIMEOUT = -8 is the expected one)."""
        return int(lib().ckks_selftest_wait(self.h, int(limit_cycles)))

    def set_stream(self, stream_ptr):
        check(lib().ckks_set_stream(self.h, stream_ptr))

    def set_fusion(self, enabled):
        check(lib().ckks_set_fusion(self.h, 1 if enabled else 0))

    def galois(self, step):
        return int(lib().ckks_galois_element(self.h, int(step)))

    def ntt(self, dev_ptr, n_rows, limbs, inverse=False):
        check(lib().ckks_ntt(self.h, dev_ptr, n_rows, limbs, 1 if inverse else 0))

    @staticmethod
    def kernel_kinds():
        n = lib().ckks_kernel_kind_count()
        return [lib().ckks_kernel_kind_name(k).decode() for k in range(n)]

    def launch_counts(self):
        names = self.kernel_kinds()
        out = np.zeros(len(names), np.uint64)
        check(lib().ckks_launch_counts(self.h, _p(out), len(names)))
        return dict(zip(names, (int(x) for x in out)))

    def profile(self, on):
        check(lib().ckks_profile_enable(self.h, 1 if on else 0))

    def int_peak(self, kind):
        """Measured integer peak: kind 0 64-bit products/s, 1 lazy forward
        butterflies/s, 2 three-product Shoup multiplies/s."""
        v = c_dbl()
        check(lib().ckks_int_peak(self.h, int(kind), ctypes.byref(v)))
        return v.value

    NTT_SLOTS = ("forward", "modup", "moddown", "rescale", "relin_rescale", "inverse")

    def autotune_ntt(self, batch=8):
        """CTAs per SM of each NTT slot chosen by measurement: ({slot: chosen},
        {slot: (ms at 2 CTAs/SM, ms at 1)})."""
        ms = np.zeros(12)
        ch = np.zeros(6, np.int32)
        check(lib().ckks_autotune_ntt(self.h, int(batch), _p(ms), _p(ch)))
        return ({n: int(ch[i]) for i, n in enumerate(self.NTT_SLOTS)},
                {n: (float(ms[i]), float(ms[6 + i])) for i, n in enumerate(self.NTT_SLOTS)})

    def set_ntt_shape(self, slot, ctas_per_sm):
        check(lib().ckks_set_ntt_shape(self.h, self.NTT_SLOTS.index(slot), int(ctas_per_sm)))

    def profile_collect(self):
        """{kind: (ms, algorithmic bytes, launches, modular multiplications)}
        since the last collect."""
        names = self.kernel_kinds()
        ms, by, mm = np.zeros(len(names)), np.zeros(len(names)), np.zeros(len(names))
        ln = np.zeros(len(names), np.uint64)
        check(lib().ckks_profile_collect2(self.h, _p(ms), _p(by), _p(mm), _p(ln), len(names)))
        return {n: (float(a), float(b), int(c), float(d))
                for n, a, b, c, d in zip(names, ms, by, ln, mm) if c}


class Keys:
    """Secret, relinearisation and Galois keys. hamming_weight > 0 draws a
    sparse secret of that weight; conjugation adds the key of X -> X^-1."""

    def __init__(self, ctx, seed, rot_steps=(), hamming_weight=0, conjugation=False,
                 public_seed=0):
        steps = np.ascontiguousarray(list(rot_steps), dtype=np.int32)
        h = c_vp()
        if hamming_weight or conjugation or public_seed:
            check(lib().ckks_keygen_ex(ctx.h, seed, int(hamming_weight),
                                       _p(steps) if len(steps) else None, len(steps),
                                       int(bool(conjugation)), int(public_seed), ctypes.byref(h)))
        else:
            check(lib().ckks_keygen(ctx.h, seed, _p(steps) if len(steps) else None, len(steps),
                                    ctypes.byref(h)))
        self.h, self.ctx = h, ctx

    def close(self):
        if self.h:
            lib().ckks_keys_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def compress(self):
        """Keep only the switching keys' b halves (seed-compressed keys)."""
        check(lib().ckks_keys_compress(self.h))

    def nbytes(self):
        n = c_sz()
        check(lib().ckks_keys_bytes(self.h, ctypes.byref(n)))
        return n.value

    def export_secret(self):
        out = np.zeros((self.ctx.n_qp, self.ctx.N), np.uint64)
        check(lib().ckks_keys_export_secret(self.h, _p(out), out.size))
        return out

    def export_switch(self, galois=0):
        out = np.zeros((self.ctx.beta_max, 2, self.ctx.n_qp, self.ctx.N), np.uint64)
        check(lib().ckks_keys_export_switch(self.h, galois, _p(out), out.size))
        return out


class Ciphertext:
    """Owns a ckks_ct handle: a batch of B ciphertexts at one level."""

    def __init__(self, ctx, h):
        self.ctx, self.h = ctx, h
        B, lv, sc = c_sz(), ctypes.c_int(), c_dbl()
        check(lib().ckks_ct_info(h, ctypes.byref(B), ctypes.byref(lv), ctypes.byref(sc)))
        self.batch, self.level, self.scale = B.value, lv.value, sc.value

    def close(self):
        if self.h:
            lib().ckks_ct_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def export(self):
        out = np.zeros((self.batch, 2, self.level + 1, self.ctx.N), np.uint64)
        check(lib().ckks_ct_export(self.h, _p(out), out.size))
        return out

    @staticmethod
    def import_(ctx, data, level, scale):
        data = np.ascontiguousarray(data, dtype=np.uint64)
        if data.ndim == 3:
            data = data[None]
        h = c_vp()
        check(lib().ckks_ct_import(ctx.h, _p(data), data.shape[0], level, scale, ctypes.byref(h)))
        return Ciphertext(ctx, h)

    def words(self):
        return self.batch * 2 * (self.level + 1) * self.ctx.N

    def export_to(self, host_ptr, cap_words):
        """Copy to caller-owned host memory (e.g. a pinned buffer)."""
        check(lib().ckks_ct_export(self.h, host_ptr, cap_words))

    @staticmethod
    def import_from(ctx, host_ptr, batch, level, scale):
        h = c_vp()
        check(lib().ckks_ct_import(ctx.h, host_ptr, batch, level, scale, ctypes.byref(h)))
        return Ciphertext(ctx, h)

    @staticmethod
    def import_from_async(ctx, host_ptr, batch, level, scale, copy_stream_ptr):
        """Copy on `copy_stream_ptr`; the library's stream waits for it."""
        h = c_vp()
        check(lib().ckks_ct_import_async(ctx.h, host_ptr, batch, level, scale, copy_stream_ptr,
                                         ctypes.byref(h)))
        return Ciphertext(ctx, h)

    def slice(self, first, count):
        h = c_vp()
        check(lib().ckks_ct_slice(self.ctx.h, self.h, first, count, ctypes.byref(h)))
        return Ciphertext(self.ctx, h)


def _out(ctx, fn, *args):
    h = c_vp()
    check(fn(*args, ctypes.byref(h)))
    return Ciphertext(ctx, h)


def encrypt(ctx, keys, values, level, seed, first_index=0):
    v = np.ascontiguousarray(values, dtype=np.float64)
    if v.ndim == 1:
        v = v[None]
    return _out(ctx, lib().ckks_encrypt, ctx.h, keys.h, _p(v), v.shape[0], v.shape[1], level,
                seed, first_index)


def decrypt(ctx, keys, ct, n=None):
    n = ctx.slots if n is None else n
    out = np.zeros((ct.batch, n))
    check(lib().ckks_decrypt(ctx.h, keys.h, ct.h, _p(out), n))
    return out


def add(ctx, a, b):
    return _out(ctx, lib().ckks_add, ctx.h, a.h, b.h)


def sub(ctx, a, b):
    return _out(ctx, lib().ckks_sub, ctx.h, a.h, b.h)


def mul_relin(ctx, keys, a, b):
    return _out(ctx, lib().ckks_mul_relin, ctx.h, keys.h, a.h, b.h)


def rescale(ctx, a):
    return _out(ctx, lib().ckks_rescale, ctx.h, a.h)


def rescale_noalloc(ctx, d_in, batch, level, d_out):
    """Rescale raw device buffers without any device allocation (see the header)."""
    check(lib().ckks_rescale_noalloc(ctx.h, d_in, batch, level, d_out))


def mul(ctx, keys, a, b):
    return _out(ctx, lib().ckks_mul, ctx.h, keys.h, a.h, b.h)


def mul_plain(ctx, a, v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    return _out(ctx, lib().ckks_mul_plain, ctx.h, a.h, _p(v), len(v))


def add_plain(ctx, a, v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    return _out(ctx, lib().ckks_add_plain, ctx.h, a.h, _p(v), len(v))


def mul_const(ctx, a, c):
    return _out(ctx, lib().ckks_mul_const, ctx.h, a.h, float(c))


def add_const(ctx, a, c):
    return _out(ctx, lib().ckks_add_const, ctx.h, a.h, float(c))


def level_down(ctx, a, level):
    return _out(ctx, lib().ckks_level_down, ctx.h, a.h, int(level))


def rotate(ctx, keys, a, step):
    return _out(ctx, lib().ckks_rotate, ctx.h, keys.h, a.h, int(step))


def rotate_hoisted(ctx, keys, a, steps):
    s = np.ascontiguousarray(list(steps), dtype=np.int32)
    hs = (c_vp * len(s))()
    check(lib().ckks_rotate_hoisted(ctx.h, keys.h, a.h, _p(s), len(s), hs))
    return [Ciphertext(ctx, c_vp(h)) for h in hs]


# ---------------------------------------------------------------- bootstrapping
def mod_raise(ctx, a, level=None):
    return _out(ctx, lib().ckks_mod_raise, ctx.h, a.h, ctx.L if level is None else level)


def conjugate(ctx, keys, a):
    return _out(ctx, lib().ckks_conjugate, ctx.h, keys.h, a.h)


def mul_monomial(ctx, a, k):
    return _out(ctx, lib().ckks_mul_monomial, ctx.h, a.h, int(k))


def mul_const_wide(ctx, a, value):
    return _out(ctx, lib().ckks_mul_const_wide, ctx.h, a.h, float(value))


def _steps(fn, h):
    n = c_sz()
    check(fn(h, None, 0, ctypes.byref(n)))
    out = np.zeros(n.value, np.int32)
    if n.value:
        check(fn(h, _p(out), n.value, ctypes.byref(n)))
    return [int(x) for x in out]


class LinearTransform:
    """z -> sum_k d_k (.) rot(z, base + k stride): diags [n_diag][N/2]
    complex, encoded for inputs at `level` with scale in_scale (0: canonical);
    form "single" (hoisted) or "double" (double hoisting)."""

    FORMS = ("single", "double")

    def __init__(self, ctx, level, base, stride, diags, g1=0, in_scale=0.0, form="single"):
        d = np.asarray(diags, dtype=complex)
        if d.ndim != 2 or d.shape[1] != ctx.slots:
            raise ValueError("diagonals must be [n_diag][N/2]")
        re = np.ascontiguousarray(d.real, dtype=np.float64)
        im = np.ascontiguousarray(d.imag, dtype=np.float64)
        h = c_vp()
        check(lib().ckks_lt_create(ctx.h, level, float(in_scale), int(base), int(stride), d.shape[0],
                                   _p(re), _p(im), int(g1), self.FORMS.index(form),
                                   ctypes.byref(h)))
        self.h, self.ctx, self.level = h, ctx, level

    def rotations(self):
        return _steps(lib().ckks_lt_rotations, self.h)

    def apply(self, keys, a):
        return _out(self.ctx, lib().ckks_lt_apply, self.ctx.h, keys.h, self.h, a.h)

    def close(self):
        if self.h:
            lib().ckks_lt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BootPlan:
    """A bootstrapping plan: BootPlan(ctx, K, degree, cts_levels, stc_levels)
    computed by the library, or BootPlan.from_parts(ctx, e, cheb, cts, stc)
    from given transforms (kept alive by the plan object)."""

    def __init__(self, ctx, K=None, degree=None, cts_levels=3, stc_levels=3, form="double",
                 _h=None, _keep=()):
        if _h is None:
            _h = c_vp()
            check(lib().ckks_boot_create(ctx.h, K, degree, cts_levels, stc_levels,
                                         LinearTransform.FORMS.index(form), ctypes.byref(_h)))
        self.h, self.ctx, self._keep = _h, ctx, list(_keep)
        e, lc, ls, nc = c_i32(), c_i32(), c_i32(), c_sz()
        check(lib().ckks_boot_info(self.h, ctypes.byref(e), ctypes.byref(lc), ctypes.byref(ls),
                                   ctypes.byref(nc)))
        self.e, self.cts_level, self.stc_level, self.n_cheb = e.value, lc.value, ls.value, nc.value

    @classmethod
    def from_parts(cls, ctx, e, cheb, cts, stc):
        cf = np.ascontiguousarray(cheb, dtype=np.float64)
        a = (c_vp * len(cts))(*[t.h for t in cts])
        b = (c_vp * len(stc))(*[t.h for t in stc])
        h = c_vp()
        check(lib().ckks_boot_create_ex(ctx.h, int(e), _p(cf), len(cf), a, len(cts), b, len(stc),
                                        ctypes.byref(h)))
        return cls(ctx, _h=h, _keep=list(cts) + list(stc))

    def rotations(self):
        return _steps(lib().ckks_boot_rotations, self.h)

    def coefficients(self):
        out = np.zeros(self.n_cheb)
        check(lib().ckks_boot_coefficients(self.h, _p(out), len(out)))
        return out

    def coeff_to_slot(self, keys, raised):
        lo, hi = c_vp(), c_vp()
        check(lib().ckks_boot_coeff_to_slot(self.ctx.h, keys.h, self.h, raised.h,
                                            ctypes.byref(lo), ctypes.byref(hi)))
        return Ciphertext(self.ctx, lo), Ciphertext(self.ctx, hi)

    def eval_mod(self, keys, a):
        return _out(self.ctx, lib().ckks_boot_eval_mod, self.ctx.h, keys.h, self.h, a.h)

    def slot_to_coeff(self, keys, lo, hi):
        return _out(self.ctx, lib().ckks_boot_slot_to_coeff, self.ctx.h, keys.h, self.h, lo.h, hi.h)

    def bootstrap(self, keys, a):
        return _out(self.ctx, lib().ckks_bootstrap, self.ctx.h, keys.h, self.h, a.h)

    def close(self):
        if self.h:
            lib().ckks_boot_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def boot_levels(ctx, n_levels, inverse, index):
    """The library's merged transform level: (base, stride, diags)."""
    b, s, n = c_i64(), c_i64(), c_sz()
    check(lib().ckks_boot_levels(ctx.h, n_levels, int(inverse), index, None, None, 0,
                                 ctypes.byref(b), ctypes.byref(s), ctypes.byref(n)))
    re = np.zeros((n.value, ctx.N // 2))
    im = np.zeros_like(re)
    check(lib().ckks_boot_levels(ctx.h, n_levels, int(inverse), index, _p(re), _p(im), re.size,
                                 ctypes.byref(b), ctypes.byref(s), ctypes.byref(n)))
    return b.value, s.value, re + 1j * im


def _descs(layers, keep):
    descs = (KanLayerDesc * len(layers))()
    for d, L in zip(descs, layers):
        b0 = L.get("b0", "product")
        if b0 not in B0_FORMS:
            raise ValueError("b0 must be 'product' or 'difference', not %r" % (b0,))
        arrs = [np.ascontiguousarray(L[k], dtype=np.float64) for k in ("coef", "w_s", "w_b")]
        cheb = np.ascontiguousarray(L.get("silu_cheb", [0.0, 0.0]), dtype=np.float64)
        stages = list(L.get("comp", [1]))
        if all(isinstance(st, (int, np.integer)) for st in stages):
            comp = np.ascontiguousarray(stages, dtype=np.int32)
            poly = plen = None
        else:  # explicit odd coefficient lists
            if any(isinstance(st, (int, np.integer)) for st in stages):
                raise ValueError("comparison stages are all f_n orders or all coefficient lists")
            comp = np.zeros(1, np.int32)
            cl = [np.ascontiguousarray(st, dtype=np.float64) for st in stages]
            poly = np.ascontiguousarray(np.concatenate(cl))
            plen = np.ascontiguousarray([len(c) for c in cl], dtype=np.int32)
            keep += [poly, plen]
        keep += arrs + [cheb, comp]
        d.n_in, d.n_out, d.G, d.k = L["n_in"], L["n_out"], L["G"], L["k"]
        d.grid_lo, d.grid_hi = L["lo"], L["hi"]
        d.coef, d.w_s, d.w_b = _p(arrs[0]), _p(arrs[1]), _p(arrs[2])
        d.R, d.silu_lo, d.silu_hi = L.get("R", 1.0), L.get("silu_lo", -1.0), L.get("silu_hi", 1.0)
        d.silu_cheb, d.silu_degree = _p(cheb), len(cheb) - 1
        d.comp, d.n_comp = _p(comp), len(comp)
        d.naive = 1 if L.get("naive") else 0
        d.comp_poly, d.comp_poly_len = _p(poly), _p(plen)
        d.n_comp_poly = 0 if poly is None else len(plen)
        d.b0_form = B0_FORMS[b0]
        bsgs = L.get("bsgs", "single")
        if bsgs not in BSGS_FORMS:
            raise ValueError("bsgs must be 'single' or 'double', not %r" % (bsgs,))
        d.bsgs_form = BSGS_FORMS[bsgs]
    return descs


B0_FORMS = {"product": 0, "difference": 1}
BSGS_FORMS = {"single": 0, "double": 1}


def comp_minimax(eps, degrees, A=1.0):
    """PolyComp stages by the library's minimax design (kan_comp_minimax):
    (list of odd coefficient arrays, taus)."""
    deg = np.ascontiguousarray(degrees, dtype=np.int32)
    coef = np.zeros(int(sum((d + 1) // 2 for d in degrees)))
    taus = np.zeros(len(degrees))
    check(lib().kan_comp_minimax(float(eps), float(A), _p(deg), len(deg), _p(coef), _p(taus)))
    out, off = [], 0
    for d in degrees:
        out.append(coef[off:off + (d + 1) // 2].copy())
        off += (d + 1) // 2
    return out, taus


FIT_METHODS = {"wls": 0, "ols": 1, "remez": 2}


def silu_fit(lo, hi, mu, sigma, degree, n_samples=10000, method="wls"):
    out = np.zeros(degree + 1)
    check(lib().kan_silu_fit(lo, hi, mu, sigma, degree, n_samples, FIT_METHODS[method], _p(out)))
    return out


def calibrate(layers, X, silu_degree, comp, fixed_range=None, n_fit_samples=10000, method="wls"):
    """Per-layer R, SiLU range and fit (Eqs. 11-12) computed by the library;
    returns copies of the layer dicts with the HE keys filled in."""
    keep = []
    descs = _descs([dict(L, comp=list(comp)) for L in layers], keep)
    X = np.ascontiguousarray(X, dtype=np.float64)
    n = len(layers)
    R, lo, hi = np.zeros(n), np.zeros(n), np.zeros(n)
    cheb = np.zeros((n, silu_degree + 1))
    fr = None if fixed_range is None else np.ascontiguousarray(fixed_range, dtype=np.float64)
    check(lib().kan_calibrate(descs, n, _p(X), X.shape[0], silu_degree, _p(fr), n_fit_samples,
                              FIT_METHODS[method], _p(R), _p(lo), _p(hi), _p(cheb)))
    out = []
    for i, L in enumerate(layers):
        L = dict(L)
        L.update(R=float(R[i]), silu_lo=float(lo[i]), silu_hi=float(hi[i]), silu_cheb=cheb[i].copy(),
                 comp=list(comp))
        out.append(L)
    return out


class Model:
    """kan_model handle; `layers` are dicts as produced for the plaintext KAN
    plus the HE keys R, silu_lo, silu_hi, silu_cheb and comp."""

    def __init__(self, ctx, layers):
        self.ctx = ctx
        self._keep = []
        descs = _descs(layers, self._keep)
        h = c_vp()
        check(lib().kan_model_create(ctx.h, descs, len(layers), ctypes.byref(h)))
        self.h = h
        self.n_layers = len(layers)

    def close(self):
        if self.h:
            lib().kan_model_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rotations(self):
        n = c_sz()
        check(lib().kan_model_rotations(self.h, None, 0, ctypes.byref(n)))
        out = np.zeros(max(n.value, 1), np.int32)
        check(lib().kan_model_rotations(self.h, _p(out), len(out), ctypes.byref(n)))
        return [int(x) for x in out[: n.value]]

    def layer_depth(self, layer):
        d = ctypes.c_int()
        check(lib().kan_model_layer_depth(self.h, layer, ctypes.byref(d)))
        return d.value

    def set_bootstrap(self, plan):
        """Refresh the batch between layers with `plan` (a BootPlan) when
        the next layer needs more levels than are left; None clears it."""
        check(lib().kan_model_set_bootstrap(self.h, plan.h if plan is not None else None))
        self._boot = plan

    def refresh_rotations(self, batch):
        """Rotation steps the packed refresh of a batch of `batch` takes."""
        n = c_sz()
        check(lib().kan_model_refresh_rotations(self.h, batch, None, 0, ctypes.byref(n)))
        out = np.zeros(n.value, np.int32)
        if n.value:
            check(lib().kan_model_refresh_rotations(self.h, batch, _p(out), n.value, ctypes.byref(n)))
        return [int(x) for x in out]

    def set_graphs(self, enabled):
        check(lib().kan_model_set_graphs(self.h, 1 if enabled else 0))

    def layer_chunks(self, layer):
        """(K, n_c): input ciphertexts per request and inputs per chunk."""
        K, n_c = ctypes.c_int(), ctypes.c_int()
        check(lib().kan_model_layer_chunks(self.h, layer, ctypes.byref(K), ctypes.byref(n_c)))
        return K.value, n_c.value

    def pack_input(self, x):
        """Rows of one request's input as the first layer takes them: the
        input itself, or K zero-padded chunks of n_c inputs."""
        x = np.asarray(x, np.float64)
        K, n_c = self.layer_chunks(0)
        if K == 1:
            return x
        xp = np.zeros(K * n_c)
        xp[: len(x)] = x
        return xp.reshape(K, n_c)


def kan_layer_eval(ctx, keys, model, layer, ct):
    return _out(ctx, lib().kan_layer_eval, ctx.h, keys.h, model.h, int(layer), ct.h)


def kan_infer(ctx, keys, model, cts):
    hs = (c_vp * len(cts))(*[c.h.value if isinstance(c.h, c_vp) else c.h for c in cts])
    return _out(ctx, lib().kan_infer, ctx.h, keys.h, model.h, hs, len(cts))


class Server:
    """kan_server handle: continuous batching of encrypted KAN requests."""

    def __init__(self, ctx, hbm_budget_bytes):
        h = c_vp()
        check(lib().kan_server_create(ctx.h, int(hbm_budget_bytes), ctypes.byref(h)))
        self.h, self.ctx = h, ctx
        self._models = []

    def close(self):
        if self.h:
            lib().kan_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_model(self, model, keys):
        mid = ctypes.c_int()
        check(lib().kan_server_add_model(self.h, model.h, keys.h, ctypes.byref(mid)))
        self._models.append((model, keys))
        return mid.value

    def submit(self, model_id, ct):
        rid = c_u64()
        check(lib().kan_server_submit(self.h, int(model_id), ct.h, ctypes.byref(rid)))
        return rid.value

    def step(self):
        n = c_sz()
        check(lib().kan_server_step(self.h, ctypes.byref(n)))
        return n.value

    def take(self, request_id):
        """The finished ciphertext, or None while the request is pending."""
        h = c_vp()
        rc = lib().kan_server_take(self.h, int(request_id), ctypes.byref(h))
        if rc == PENDING:
            return None
        check(rc)
        return Ciphertext(self.ctx, h)

    def status(self):
        v = [c_sz() for _ in range(6)]
        check(lib().kan_server_status(self.h, *[ctypes.byref(x) for x in v]))
        return dict(zip(("waiting", "active", "finished", "hbm_in_use", "hbm_peak",
                         "hbm_measured_peak"), (x.value for x in v)))

    def footprint(self, model_id):
        """Measured device bytes one request of the model needs."""
        v = c_sz()
        check(lib().kan_server_footprint(self.h, int(model_id), ctypes.byref(v)))
        return v.value
