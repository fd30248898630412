"""Per-layer HE parameters from a calibration set (test infrastructure only).

For every layer: the SiLU range and weighted least-squares fit of Eqs. 11-12
on the layer's inputs, and the comparison bound R of Algorithm 2 (inputs are
represented in [-R, R]; reading: R is 1.1 times the half-width that keeps
|x - t_m| / (2R) <= 1 for every calibration input x and knot t_m).

Reading: "the layer's inputs" are the values the encrypted network computes,
i.e. the HE-friendly FP64 KAN (fitted SiLU, PolyComp indicators) with the
layers before it already calibrated; the soft comparisons shift hidden
activations, and a range taken from the exact KAN would leave the encrypted
network's values outside the fit, where the polynomial's evaluation
amplifies the CKKS noise. Layer 0's inputs are the data themselves.
"""
import numpy as np

from .kan_plain import knots, layer_forward
from .silu_fit import fit_silu, layer_stats, silu_range


def calibrate(model, X, silu_degree, comp, fixed_range=None, n_samples=10000, method="wls"):
    h = np.asarray(X, dtype=np.float64)
    out = []
    for layer in model:
        a = h
        mu, sigma, mn, mx = layer_stats(a)
        lo, hi = fixed_range if fixed_range is not None else silu_range(mu, sigma, mn, mx)
        L = dict(layer)
        L["silu_lo"], L["silu_hi"] = float(lo), float(hi)
        L["silu_cheb"] = fit_silu(lo, hi, mu, sigma, silu_degree, n_samples, method)
        L["silu_stats"] = (mu, sigma, mn, mx)
        t = knots(layer)
        L["R"] = 1.1 * (np.abs(a).max() + np.abs(t).max()) / 2.0
        L["comp"] = list(comp)
        out.append(L)
        h = layer_forward(L, h, "poly", "poly")
    return out
