"""ctypes loader for the oracle's C core (test infrastructure only).

`build()` compiles `ckks_oracle.c` with gcc into `liboracle.so` next to it.
Floating-point contraction is disabled so the FP64 encoder rounds the same
way on every IEEE-754 host.
"""
import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ckks_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")

_lib = None


def build(force=False):
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = ctypes.CDLL(_SO)
    u64, i64, i32, u32, dbl, vp = (ctypes.c_uint64, ctypes.c_int64, ctypes.c_int,
                                   ctypes.c_uint32, ctypes.c_double, ctypes.c_void_p)
    sig = {
        "or_mulmod": (u64, [u64, u64, u64]),
        "or_powmod": (u64, [u64, u64, u64]),
        "or_is_prime": (i32, [u64]),
        "or_gen_chain": (i32, [i32, i32, i32, i32, i32, i32, vp, vp, vp]),
        "or_find_psi": (u64, [u64, i32]),
        "or_ntt_naive": (None, [vp, vp, i32, u64, u64]),
        "or_ntt_forward": (None, [vp, i32, u64, u64]),
        "or_ntt_inverse": (None, [vp, i32, u64, u64]),
        "or_negacyclic_mul": (None, [vp, vp, vp, i32, u64]),
        "or_automorphism_coef": (None, [vp, vp, i32, u64, u64]),
        "or_automorphism_ntt": (None, [vp, vp, i32, u64]),
        "or_encode": (i32, [vp, u64, i32, dbl, vp]),
        "or_decode": (None, [vp, i32, vp, u64]),
        "or_chacha20_quarter": (None, [vp]),
        "or_chacha20_block": (None, [vp, u32, vp, vp]),
        "or_stream_word32": (u32, [u64, u32, u64, u64]),
        "or_sample_ternary": (None, [u64, i32, vp]),
        "or_sample_cbd": (None, [u64, u64, i32, vp]),
        "or_sample_uniform": (None, [u64, u64, u32, u64, i32, vp]),
        "or_ctx_create": (vp, [i32, i32, i32, i32, i32, i32]),
        "or_ctx_destroy": (None, [vp]),
        "or_ctx_info": (i32, [vp, vp, vp, vp]),
        "or_ntt_limb": (None, [vp, vp, i32, i32]),
        "or_keygen_secret": (None, [vp, u64, vp, vp]),
        "or_target_secret": (None, [vp, vp, u64, vp]),
        "or_keygen_switch": (None, [vp, u64, vp, vp, u64, vp]),
        "or_keygen_switch_pub": (None, [vp, u64, u64, vp, vp, u64, vp]),
        "or_encode_plain": (i32, [vp, vp, u64, i32, dbl, vp]),
        "or_encrypt": (i32, [vp, vp, vp, u64, i32, u64, u64, vp]),
        "or_decrypt": (None, [vp, vp, vp, i32, dbl, vp, u64]),
        "or_add": (None, [vp, vp, vp, i32, i32, i32, vp]),
        "or_mul_plain": (None, [vp, vp, vp, i32, i32, vp]),
        "or_mul_int": (None, [vp, vp, i64, i32, i32, vp]),
        "or_add_int": (None, [vp, vp, i64, i32]),
        "or_tensor": (None, [vp, vp, vp, i32, vp]),
        "or_automorphism_polys": (None, [vp, vp, i32, u64, vp]),
        "or_rescale": (None, [vp, vp, i32, i32, vp]),
        "or_modup": (None, [vp, vp, i32, vp]),
        "or_keyswitch_ext": (None, [vp, vp, i32, vp, u64, vp]),
        "or_relin_rescale": (None, [vp, vp, vp, i32, vp, vp]),
        "or_div_p_ql": (None, [vp, vp, vp, i32, vp]),
        "or_key_product": (None, [vp, vp, i32, vp, u64, vp]),
        "or_qp_mul_plain_acc": (None, [vp, vp, vp, i32, vp]),
        "or_qp_lift": (None, [vp, vp, i32, u64, vp, vp]),
        "or_encode_complex": (i32, [vp, vp, u64, i32, dbl, vp]),
        "or_decode_complex": (None, [vp, i32, vp, vp, u64]),
        "or_encode_plain_complex": (i32, [vp, vp, vp, u64, i32, dbl, vp]),
        "or_mod_raise": (None, [vp, vp, i32, vp]),
        "or_sample_sparse_ternary": (None, [u64, i32, i32, vp]),
        "or_keygen_secret_sparse": (None, [vp, u64, i32, vp, vp]),
        "or_ext_rows": (u64, [vp, i32]),
        "or_galois_elt": (u64, [vp, i64]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def ptr(a):
    """Address of a C-contiguous numpy array."""
    assert a.flags["C_CONTIGUOUS"], "array must be C-contiguous"
    return a.ctypes.data
