"""FP64 plaintext KAN (test infrastructure only).

Two forms of the same network:

* exact — Eqs. 1-5: phi(x) = w_b * silu(x) + w_s * sum_m c_m B_{m,k}(x) with
  the Cox-de Boor recursion (Eqs. 2-3; half-open intervals t_m <= x < t_{m+1},
  zero outside the extended grid);
* HE-friendly ("HEF") — the same network with silu replaced by the fitted
  Chebyshev polynomial and each order-0 indicator B_{m,0} replaced by the
  product of two comparison polynomials (Algorithm 2, lines 4-6), keeping the
  recursion of Algorithm 2 (lines 7-14) otherwise unchanged.

A model is a list of layer dicts with keys:
  n_in, n_out, G (grid intervals), k (order), lo, hi (grid range),
  coef [n_out, n_in, G+k], w_s [n_out, n_in], w_b [n_out, n_in]
and, for the HE-friendly form,
  R (comparison bound), silu_lo, silu_hi, silu_cheb (Chebyshev coefficients),
  comp (composite stages: orders n for f_n, or odd coefficient lists),
  b0 ("product", Algorithm 2's form, or "difference").
"""
import numpy as np


def knots(layer):
    """Extended uniform grid: t_m = lo + (m - k) h, m = 0..G+2k."""
    G, k, lo, hi = layer["G"], layer["k"], layer["lo"], layer["hi"]
    h = (hi - lo) / G
    return lo + (np.arange(G + 2 * k + 1) - k) * h


def silu(x):
    """Eq. 5."""
    return x / (1.0 + np.exp(-x))


def bspline_exact(x, t, k):
    """Cox-de Boor, Eqs. 2-3. x: [...]; returns [..., len(t) - 1 - k]."""
    x = np.asarray(x, dtype=np.float64)[..., None]
    B = ((t[:-1] <= x) & (x < t[1:])).astype(np.float64)
    for j in range(1, k + 1):
        left = (x - t[: -(j + 1)]) / (t[j:-1] - t[: -(j + 1)]) * B[..., :-1]
        right = (t[j + 1:] - x) / (t[j + 1:] - t[1:-j]) * B[..., 1:]
        B = left + right
    return B


# ------------------------------------------------------------------ comparison
def fn_coeffs(n):
    """Odd monomial coefficients of f_n(x) = sum_{i=0}^n 4^-i C(2i,i) x (1-x^2)^i.

    Returns c with f_n(x) = sum_l c[l] x^(2l+1). Each coefficient is a dyadic
    rational computed exactly, so it is an exact double.
    """
    from fractions import Fraction
    from math import comb
    c = [Fraction(0)] * (n + 1)
    for i in range(n + 1):
        w = Fraction(comb(2 * i, i), 4 ** i)
        for l in range(i + 1):
            c[l] += w * comb(i, l) * (-1) ** l
    return [float(v) for v in c]


def eval_odd(x, c):
    return sum(cl * x ** (2 * l + 1) for l, cl in enumerate(c))


def stage_coeffs(stage):
    """Odd monomial coefficients of one composite stage: an order n names
    f_n; a sequence gives the coefficients themselves (a minimax stage)."""
    if isinstance(stage, (int, np.integer)):
        return fn_coeffs(int(stage))
    return [float(v) for v in stage]


def polycomp0(a, stages):
    """PolyComp(a, 0) ~ (1 + sign(a)) / 2 via the composite of the stages
    (f_n by order, or explicit odd coefficient lists), first stage first."""
    u = np.asarray(a, dtype=np.float64)
    for st in stages:
        u = eval_odd(u, stage_coeffs(st))
    return 0.5 + 0.5 * u


def bspline_hef(x, t, k, R, stages, b0="product"):
    """Algorithm 2 on plaintext values: soft order-0 indicators, same recursion.

    b0 = "product": B_{m,0} = PolyComp(x - t_m) PolyComp(t_{m+1} - x) as in
    Algorithm 2. b0 = "difference": B_{m,0} = s_m - s_{m+1} with
    s_m = PolyComp(x - t_m), one comparison per knot and no product; the two
    agree for exact comparisons (PolyComp(-a) = 1 - PolyComp(a) since f is
    odd, and s_m s_{m+1} = s_{m+1} for exact steps at t_m < t_{m+1})."""
    x = np.asarray(x, dtype=np.float64)[..., None]
    if b0 == "difference":
        s = polycomp0((x - t) / (2.0 * R), stages)
        B = s[..., :-1] - s[..., 1:]
    else:
        s1 = polycomp0((x - t[:-1]) / (2.0 * R), stages)
        s2 = polycomp0((t[1:] - x) / (2.0 * R), stages)
        B = s1 * s2
    for j in range(1, k + 1):
        left = (x - t[: -(j + 1)]) / (t[j:-1] - t[: -(j + 1)]) * B[..., :-1]
        right = (t[j + 1:] - x) / (t[j + 1:] - t[1:-j]) * B[..., 1:]
        B = left + right
    return B


def cheb_eval(x, lo, hi, a):
    y = (2.0 * x - (lo + hi)) / (hi - lo)
    return np.polynomial.chebyshev.chebval(y, a)


# ------------------------------------------------------------------ forward
def layer_forward(layer, x, silu_mode="exact", basis_mode="exact"):
    """x: [batch, n_in] -> [batch, n_out]."""
    t = knots(layer)
    if silu_mode == "exact":
        sx = silu(x)
    else:
        sx = cheb_eval(x, layer["silu_lo"], layer["silu_hi"], layer["silu_cheb"])
    if basis_mode == "exact":
        B = bspline_exact(x, t, layer["k"])
    else:
        B = bspline_hef(x, t, layer["k"], layer["R"], layer["comp"], layer.get("b0", "product"))
    base = sx @ layer["w_b"].T
    spline = np.einsum("bim,oim,oi->bo", B, layer["coef"], layer["w_s"])
    return base + spline


def forward(model, x, silu_mode="exact", basis_mode="exact", collect=False):
    acts = []
    h = np.asarray(x, dtype=np.float64)
    for layer in model:
        acts.append(h)
        h = layer_forward(layer, h, silu_mode, basis_mode)
    return (h, acts) if collect else h
