"""Writes tests/golden/boot_digest.json: SHA-256 digests, limb by limb, of one
CKKS bootstrap at full size, computed by the oracle alone (test
infrastructure; nothing here touches the CUDA library).

Case: N = 2^16, a 60-bit q0 under 28 primes of 50 bits, alpha = 5 special
primes of 60 bits; sparse ternary secret of weight 192 (key seed 7);
K = 30, EvalMod of degree 255; three merged levels of double-hoisted
transforms each way (the bench's bootstrapping workload). Input: the 32768
slots uniform on [-1, 1] from numpy's default_rng(6), encrypted at level 0
(seed 9, object 0). The transforms' diagonals come out the same on every
machine (correctly rounded roots, products rounded once each), but numpy's
Chebyshev interpolation need not, so the file stores the EvalMod
coefficients the oracle used; a test rebuilds the plan from them.

Run: python tests/golden/make_boot_digest.py (about ten minutes and ten GB
of host memory for the keys).
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import boot as OB, ckks as O  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "boot_digest.json")
PARAMS = dict(log_n=16, n_scale=28, n_special=5, q0_bits=60, scale_bits=50)
K, DEGREE, LEVELS, FORM, H, KEY_SEED, ENC_SEED, INPUT_SEED = 30, 255, 3, "double", 192, 7, 9, 6


def limb_digests(data):
    d = np.ascontiguousarray(data, dtype="<u8")
    return [[hashlib.sha256(d[p, t].tobytes()).hexdigest() for t in range(d.shape[1])]
            for p in range(d.shape[0])]


def main():
    t0 = time.time()
    ctx = O.Ctx(O.Params(**PARAMS))
    plan = OB.Plan(ctx, K, DEGREE, LEVELS, LEVELS, form=FORM)
    keys = OB.BootKeys(ctx, KEY_SEED, plan.steps(ctx), h=H)
    z = np.random.default_rng(INPUT_SEED).uniform(-1, 1, ctx.slots)
    ct = O.encrypt(ctx, keys, z, 0, ENC_SEED, 0)
    raised = OB.mod_raise(ctx, ct)
    lo, hi = OB.coeff_to_slot(ctx, keys, raised, plan.K, plan.cts)
    lo = OB.kan_he.eval_cheb(ctx, keys, lo, plan.cheb)
    hi = OB.kan_he.eval_cheb(ctx, keys, hi, plan.cheb)
    stc_level = min(lo.level, hi.level)
    out = OB.slot_to_coeff(ctx, keys, lo, hi, plan.stc)
    err = float(np.abs(O.decrypt(ctx, keys, out) - z).max())
    res = dict(params=PARAMS, K=K, degree=DEGREE, levels=LEVELS, form=FORM, hamming=H,
               key_seed=KEY_SEED, enc_seed=ENC_SEED, input_seed=INPUT_SEED,
               e=OB.mod_exponent(ctx, K), cheb=[float(v) for v in plan.cheb],
               cts_level=ctx.L, stc_level=stc_level, steps=plan.steps(ctx),
               level=out.level, scale=out.scale, limbs=limb_digests(out.data),
               max_abs_error=err, oracle_seconds=round(time.time() - t0, 1))
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1, sort_keys=True)
        f.write("\n")
    print("level", out.level, "error %.2e" % err, "oracle", res["oracle_seconds"], "s")


if __name__ == "__main__":
    main()
