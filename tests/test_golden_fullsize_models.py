"""The full-size golden file is self-consistent (CPU): for every case, the
seeded weights and the stored calibration rebuild the model whose digest
the oracle's output digests were computed with. On a machine whose seeded
weights differ, this fails here rather than as a word mismatch on the GPU."""
import json
import os
import sys

import pytest

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLD)
import make_fullsize_digests as D  # noqa: E402

with open(os.path.join(GOLD, "fullsize_digests.json")) as f:
    GOLDEN = json.load(f)


@pytest.mark.parametrize("name", sorted(GOLDEN))
def test_stored_calibration_rebuilds_the_digested_model(name):
    ref = GOLDEN[name]
    params, m, x, level, scope = D.rebuild(name, ref)
    assert D.weights_digest(m) == ref["weights_sha256"]
    assert D.model_digest(m) == ref["model_sha256"]
    assert len(x) == ref["n_input_cts"] and len(ref["limbs"]) == 2
    assert all(len(p) == ref["level"] + 1 for p in ref["limbs"])
