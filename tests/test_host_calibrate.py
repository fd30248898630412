"""Host-side model preparation of the library (no GPU work) against the
oracle: SiLU range (Eq. 11), weighted least-squares fit (Eq. 12), the
comparison bound R, and the plaintext forward pass it runs on."""
import numpy as np
import pytest

from oracle import calibrate as OC, silu_fit as OF
from paper_2409_07751_gb300 import workloads as W


@pytest.fixture(scope="module")
def G():
    from paper_2409_07751_gb300 import build, ckks
    build.build()
    return ckks


@pytest.mark.parametrize("args", [(-4.0, 4.0, 0.1, 0.6, 15), (-1.0, 1.0, 0.0, 0.58, 27),
                                  (-12.4, 14.74, 0.5, 5.0, 10)])
def test_silu_fit_matches_oracle(G, args):
    lo, hi, mu, sig, d = args
    a = G.silu_fit(lo, hi, mu, sig, d, 4000)
    ref = OF.fit_silu(lo, hi, mu, sig, d, 4000)
    assert np.abs(a - ref).max() < 1e-8


@pytest.mark.parametrize("name,n_in", [("kan_4_8_4_1", 4), ("kan_2_5_1", 2)])
def test_calibrate_matches_oracle(G, name, n_in):
    model = W.make_model(name)
    X = W.uniform_inputs(300, n_in)
    fixed = (-4.0, 4.0) if name == "kan_2_5_1" else None
    g = G.calibrate(model, X, 15, [3], fixed_range=fixed, n_fit_samples=3000)
    o = OC.calibrate(model, X, 15, [3], fixed_range=fixed, n_samples=3000)
    for gl, ol in zip(g, o):
        assert abs(gl["R"] - ol["R"]) < 1e-12 * ol["R"]
        assert abs(gl["silu_lo"] - ol["silu_lo"]) < 1e-12
        assert abs(gl["silu_hi"] - ol["silu_hi"]) < 1e-12
        assert np.abs(gl["silu_cheb"] - ol["silu_cheb"]).max() < 1e-8
