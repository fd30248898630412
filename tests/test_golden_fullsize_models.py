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


def test_boot_digest_file_matches_its_plan():
    """The stored full-size bootstrap case: the rotation steps, exponent and
    levels the oracle recomputes here from the stored parameters, and the
    stored EvalMod coefficients of the stated degree."""
    from oracle import boot as OB, ckks as O
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "boot_digest.json")
    with open(path) as f:
        d = json.load(f)
    p = d["params"]
    ctx = O.Ctx(O.Params(p["log_n"], p["n_scale"], p["n_special"], q0_bits=p["q0_bits"],
                         scale_bits=p["scale_bits"]))
    steps = set()
    for inverse in (True, False):
        for lt in OB.transform_levels(ctx, d["levels"], inverse, d["form"]):
            steps |= set(lt.steps(ctx.slots))
    assert sorted(steps) == d["steps"]
    assert d["e"] == OB.mod_exponent(ctx, d["K"])
    assert len(d["cheb"]) == d["degree"] + 1 and d["cts_level"] == ctx.L
    assert d["stc_level"] == ctx.L - d["levels"] - 2 - 9 and d["level"] == d["stc_level"] - d["levels"]
    assert len(d["limbs"]) == 2 and len(d["limbs"][0]) == d["level"] + 1
    assert d["max_abs_error"] < 1e-3
