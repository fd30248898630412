"""Per-layer HE parameters from a calibration set (test infrastructure only).

For every layer: the SiLU range and weighted least-squares fit of Eqs. 11-12
on the layer's inputs under the exact FP64 KAN, and the comparison bound R
of Algorithm 2 (inputs are represented in [-R, R]; reading: R is 1.1 times
the half-width that keeps |x - t_m| / (2R) <= 1 for every calibration input
x and knot t_m).
"""
import numpy as np

from .kan_plain import forward, knots
from .silu_fit import fit_silu, layer_stats, silu_range


def calibrate(model, X, silu_degree, comp, fixed_range=None, n_samples=10000, method="wls"):
    _, acts = forward(model, X, collect=True)
    out = []
    for layer, a in zip(model, acts):
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
    return out
