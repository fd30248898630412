"""Writes tests/golden/fullsize_digests.json: SHA-256 digests, limb by limb,
of encrypted KAN outputs at the configurations' full sizes, computed by the
oracle alone (test infrastructure; nothing here touches the CUDA library).

Cases (N = 2^16, q0 + 36 x 40-bit primes; seeds of the workloads module):
  c2     [4,8,4,1], G=5, k=3, SiLU degree 27, the minimax comparison of
         degrees 7 and 15 (eps 0.12) in the difference form of B_{m,0}, digit
         layout alpha = 5 with 48-bit special primes (the batched bench's
         configuration): the whole three-layer inference of input 0 at level 36;
  c2_f3  the same network with comparison f_3 in the product form;
  c3     [784,64,10], G=5, k=3 on the 28x28 blob images, SiLU degree 15,
         comparison f_3^4, alpha = 4: layer 0 of image 0 (BSGS over n' = 8192);
  c4     [3072,64,10], G=10, k=3 on the 3x32x32 images, SiLU degree 15,
         comparison f_3^4, alpha = 4: layer 0 of image 0, split into two
         ciphertexts of 2048 inputs (BSGS over n' = 32768, chunk sum).

Each case also stores what the oracle calibrated (per layer R, the SiLU
range and Chebyshev coefficients, the comparison stages), the encrypted input
rows, a digest of the seeded weights and a digest of the whole model: the
calibration's least squares, statistics and minimax design round differently
on other machines (LAPACK, libm), so a test rebuilds the model from the
seeded weights and these stored values rather than recalibrating. `--describe`
adds these fields to the cases already in the file without rerunning them
(the model digest proves the stored values are the digested model's). Run: python tests/golden/make_fullsize_digests.py [case ...]
(the oracle needs tens of minutes per case; cases run in parallel
processes). The Galois keys are generated when a rotation first needs them
and only a few are kept, so a case fits in a few GB of host memory.
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

from oracle import calibrate, ckks as O, kan_he, polycomp  # noqa: E402
from paper_2409_07751_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fullsize_digests.json")


def case_setup(name, calibrate_model=True):
    """(params kwargs, calibrated model, input rows, input level, scope);
    calibrate_model=False returns the seeded model uncalibrated."""
    cal = calibrate.calibrate if calibrate_model else (lambda model, *a, **k: [dict(L) for L in model])
    if name == "c2":
        model = [dict(L, b0="difference") for L in W.make_model("kan_4_8_4_1")]
        Xcal = W.uniform_inputs(256, 4, seed=W.SEED_INPUTS + 1000)
        m = cal(model, Xcal, 27, polycomp.composite(0.12, (7, 15))[0])
        x = W.uniform_inputs(64, 4, seed=W.SEED_INPUTS)[:1]
        return dict(log_n=16, n_scale=36, n_special=5, p_bits=48), m, x, 36, "network"
    if name == "c2_f3":
        model = W.make_model("kan_4_8_4_1")
        Xcal = W.uniform_inputs(256, 4, seed=W.SEED_INPUTS + 1000)
        m = cal(model, Xcal, 27, [3])
        x = W.uniform_inputs(64, 4, seed=W.SEED_INPUTS)[:1]
        return dict(log_n=16, n_scale=36, n_special=5, p_bits=48), m, x, 36, "network"
    if name == "c3":
        model = W.make_model("kan_784_64_10")
        X = W.blob_images(66)
        m = cal(model, X[2:], 15, [3, 3, 3, 3])
        return dict(log_n=16, n_scale=36, n_special=4), m, X[:1], 36, "layer0"
    if name == "c4":
        model = W.make_model("kan_3072_64_10")
        X = W.cifar_like_images(34)
        m = cal(model, X[2:], 15, [3, 3, 3, 3])
        K, n_c = 2, 2048
        xp = np.pad(X[0], (0, K * n_c - 3072))
        return (dict(log_n=16, n_scale=36, n_special=4), m,
                np.stack([xp[c * n_c:(c + 1) * n_c] for c in range(K)]), 36, "layer0")
    raise KeyError(name)


def model_digest(m):
    h = hashlib.sha256()
    for L in m:
        for key in ("n_in", "n_out", "G", "k", "lo", "hi", "R", "silu_lo", "silu_hi"):
            h.update(np.float64(L[key]).tobytes())
        for key in ("coef", "w_s", "w_b", "silu_cheb"):
            h.update(np.ascontiguousarray(L[key], dtype=np.float64).tobytes())
        comp = L["comp"]
        if all(isinstance(st, (int, np.integer)) for st in comp):
            h.update(np.asarray(comp, dtype=np.int64).tobytes())
        else:
            for st in comp:
                h.update(np.asarray([len(st)], dtype=np.int64).tobytes())
                h.update(np.ascontiguousarray(st, dtype=np.float64).tobytes())
        h.update(str(L.get("b0", "product")).encode())
    return h.hexdigest()


def weights_digest(m):
    h = hashlib.sha256()
    for L in m:
        for key in ("coef", "w_s", "w_b"):
            h.update(np.ascontiguousarray(L[key], dtype=np.float64).tobytes())
    return h.hexdigest()


def describe(name):
    """The stored values a test needs to rebuild case `name` exactly."""
    params, m, x, level, scope = case_setup(name)
    layers = []
    for L in m:
        comp = L["comp"]
        layers.append(dict(
            R=float(L["R"]), silu_lo=float(L["silu_lo"]), silu_hi=float(L["silu_hi"]),
            silu_cheb=[float(v) for v in L["silu_cheb"]], b0=L.get("b0", "product"),
            comp=[int(st) if isinstance(st, (int, np.integer)) else [float(v) for v in st]
                  for st in comp]))
    return dict(calibration=layers, inputs=[[float(v) for v in row] for row in np.asarray(x)],
                weights_sha256=weights_digest(m), model_sha256=model_digest(m))


def rebuild(name, stored):
    """(params, model, input rows, level, scope) from the seeded weights and
    the stored calibration; the caller checks the digests."""
    params, m, x, level, scope = case_setup(name, calibrate_model=False)
    for L, c in zip(m, stored["calibration"]):
        L.update(R=c["R"], silu_lo=c["silu_lo"], silu_hi=c["silu_hi"],
                 silu_cheb=np.array(c["silu_cheb"]), b0=c["b0"],
                 comp=[st if isinstance(st, int) else list(st) for st in c["comp"]])
    return params, m, np.array(stored["inputs"]), level, scope


def limb_digests(data):
    """data: [2][l][N] uint64 -> [[sha256 per limb] per polynomial]."""
    d = np.ascontiguousarray(data, dtype="<u8")
    return [[hashlib.sha256(d[p, t].tobytes()).hexdigest() for t in range(d.shape[1])]
            for p in range(d.shape[0])]


class LazyGaloisKeys:
    """Galois keys of the allowed elements, generated on first use; at most
    `keep` are held at once (a key at N = 2^16 is a few hundred MB)."""

    def __init__(self, keys, elements, keep=6):
        self.keys, self.allowed, self.keep = keys, set(elements), keep
        self.cache = {}

    def __contains__(self, g):
        return g in self.allowed

    def __getitem__(self, g):
        if g not in self.allowed:
            raise KeyError(g)
        if g not in self.cache:
            if len(self.cache) >= self.keep:
                self.cache.pop(next(iter(self.cache)))
            self.cache[g] = self.keys._switch_key(g)
        v = self.cache.pop(g)
        self.cache[g] = v  # most recently used last
        return v


def run_case(name):
    t0 = time.time()
    params, m, x, level, scope = case_setup(name)
    ctx = O.Ctx(O.Params(**params))
    rots = kan_he.model_rotations(m, ctx.slots)
    keys = O.Keys(ctx, W.SEED_KEYS, rot_steps=())
    keys.galois = LazyGaloisKeys(keys, {ctx.galois(t) for t in rots} - {1})
    cts = [O.encrypt(ctx, keys, x[c], level, W.SEED_ENC, c) for c in range(len(x))]
    if scope == "network":
        out = kan_he.infer(ctx, keys, cts[0] if len(cts) == 1 else cts, m)
    elif len(cts) == 1:
        out = kan_he.layer_eval(ctx, keys, cts[0], m[0])
    else:
        out = kan_he.layer_eval_chunked(ctx, keys, cts, m[0])
    return name, dict(
        params=params, scope=scope, input_level=level, n_input_cts=len(cts),
        level=out.level, scale=out.scale, limbs=limb_digests(out.data),
        oracle_seconds=round(time.time() - t0, 1), **describe(name))


def main(names):
    import multiprocessing as mp
    res = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            res = json.load(f)
    with mp.get_context("spawn").Pool(len(names)) as pool:
        for name, r in pool.imap_unordered(run_case, names):
            res[name] = r
            print(name, "level", r["level"], "oracle", r["oracle_seconds"], "s", flush=True)
            with open(OUT, "w") as f:
                json.dump(res, f, indent=1, sort_keys=True)
                f.write("\n")


def main_describe():
    with open(OUT) as f:
        res = json.load(f)
    for name, r in res.items():
        d = describe(name)
        if d["model_sha256"] != r["model_sha256"]:
            raise SystemExit("%s: this machine calibrates another model than the digested one" % name)
        r.update(d)
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    if sys.argv[1:] == ["--describe"]:
        main_describe()
    else:
        main(sys.argv[1:] or ["c2", "c2_f3", "c3", "c4"])
