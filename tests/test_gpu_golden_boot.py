"""One CKKS bootstrap at full size (N = 2^16, 29 limbs, sparse secret of
weight 192, EvalMod degree 255, three double-hoisted transform levels each
way) against the oracle's ciphertext, limb by limb (SHA-256 digests in
tests/golden/boot_digest.json, written by make_boot_digest.py from the
oracle alone). The plan is rebuilt here from the oracle's transform levels
(the same bits on every machine) and the stored EvalMod coefficients; the
keys and the input ciphertext come from the same seeds on the GPU."""
import hashlib
import json
import os

import numpy as np
import pytest

from oracle import boot as OB, ckks as O

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "boot_digest.json")


@pytest.fixture(scope="module")
def G():
    from paper_2409_07751_gb300 import build, ckks
    build.build()
    return ckks


def test_bootstrap_full_size_matches_the_oracle(G):
    with open(GOLD) as f:
        d = json.load(f)
    p = d["params"]
    octx = O.Ctx(O.Params(p["log_n"], p["n_scale"], p["n_special"], q0_bits=p["q0_bits"],
                          scale_bits=p["scale_bits"]))
    gctx = G.Context(p["log_n"], p["n_scale"], p["n_special"], q0_bits=p["q0_bits"],
                     scale_bits=p["scale_bits"])
    cts = OB.transform_levels(octx, d["levels"], True, d["form"])
    stc = OB.transform_levels(octx, d["levels"], False, d["form"])
    steps = set()
    for lt in cts + stc:
        steps |= set(lt.steps(octx.slots))
    assert sorted(steps) == d["steps"]
    g_cts = [G.LinearTransform(gctx, d["cts_level"] - i, lt.base, lt.stride, lt.diags, g1=lt.g1,
                               in_scale=octx.delta[0] if i == 0 else 0.0, form=lt.form)
             for i, lt in enumerate(cts)]
    g_stc = [G.LinearTransform(gctx, d["stc_level"] - i, lt.base, lt.stride, lt.diags, g1=lt.g1,
                               form=lt.form)
             for i, lt in enumerate(stc)]
    gp = G.BootPlan.from_parts(gctx, d["e"], d["cheb"], g_cts, g_stc)
    keys = G.Keys(gctx, d["key_seed"], d["steps"], hamming_weight=d["hamming"], conjugation=True)
    z = np.random.default_rng(d["input_seed"]).uniform(-1, 1, gctx.slots)
    ct = G.encrypt(gctx, keys, z, 0, d["enc_seed"], 0)
    out = gp.bootstrap(keys, ct)
    assert out.level == d["level"] and out.scale == d["scale"]
    data = np.ascontiguousarray(out.export()[0], dtype="<u8")
    got = [[hashlib.sha256(data[k, t].tobytes()).hexdigest() for t in range(data.shape[1])]
           for k in range(2)]
    assert got == d["limbs"]
    assert np.abs(G.decrypt(gctx, keys, out, gctx.slots)[0] - z).max() < 1e-3
