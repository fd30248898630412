"""Word-for-word parity at the configurations' full sizes (N = 2^16, the
full 37-limb chain): the CUDA path's output ciphertexts must have the same
SHA-256 digest, limb by limb, as the oracle's, stored in
tests/golden/fullsize_digests.json by tests/golden/make_fullsize_digests.py
(an oracle-only script; the oracle needs tens of minutes per case, so its
words are stored as digests). Cases:

  c2  [4,8,4,1], alpha = 5 with 48-bit special primes, the bench's minimax
      comparison in the difference form: the whole network;
  c2_f3  the same network with the comparison f_3 in the product form;
  c3  [784,64,10]: layer 0, BSGS plans over n' = 8192 and n' = 1024;
  c4  [3072,64,10]: layer 0 in two ciphertexts of 2048 inputs, BSGS over
      n' = 32768 and the chunk sum.

Both sides get the same model: the seeded weights (checked by their digest)
with the calibration the oracle computed, stored beside the digests (a
calibration rerun on another machine rounds differently), checked by the
whole model's digest; the same input rows, keys (seed 1) and encryptions
(seed 2, index = chunk)."""
import json
import os
import sys

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLD)
import make_fullsize_digests as D  # noqa: E402
from paper_2409_07751_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

with open(os.path.join(GOLD, "fullsize_digests.json")) as f:
    GOLDEN = json.load(f)


@pytest.fixture(scope="module")
def G():
    from paper_2409_07751_gb300 import build, ckks
    build.build()
    return ckks


@pytest.mark.parametrize("name", ["c2", "c2_f3", "c3", "c4"])
def test_fullsize_output_words_match_oracle_digests(G, name):
    ref = GOLDEN[name]
    params, m, x, level, scope = D.rebuild(name, ref)
    assert params == ref["params"] and scope == ref["scope"] and level == ref["input_level"]
    assert D.weights_digest(m) == ref["weights_sha256"], "the seeded weights differ on this machine"
    assert D.model_digest(m) == ref["model_sha256"]
    ctx = G.Context(params["log_n"], params["n_scale"], params["n_special"],
                    p_bits=params.get("p_bits", 60))
    gm = G.Model(ctx, m)
    keys = G.Keys(ctx, W.SEED_KEYS, gm.rotations())
    ct = G.encrypt(ctx, keys, np.asarray(x), level, W.SEED_ENC, 0)
    assert ct.batch == ref["n_input_cts"]
    if scope == "network":
        out = G.kan_infer(ctx, keys, gm, [ct])
    else:
        out = G.kan_layer_eval(ctx, keys, gm, 0, ct)
    assert out.batch == 1
    assert out.level == ref["level"] and out.scale == ref["scale"]
    got = D.limb_digests(out.export()[0])
    bad = [(p, t) for p in range(2) for t in range(out.level + 1)
           if got[p][t] != ref["limbs"][p][t]]
    assert not bad, "limbs differing from the oracle: %s" % bad[:8]
