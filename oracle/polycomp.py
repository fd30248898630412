"""PolyComp by composite minimax polynomials (test infrastructure only).

Algorithm 2 builds the order-0 B-spline indicators from PolyComp(a, 0), which
the paper evaluates with the composite minimax polynomials of Lee et al.
(2021) without giving their degrees. The construction here (a reading):

* the composite approximates sign(a) on [-1, -eps] u [eps, 1] (eps the width
  left to the transition): PolyComp's range. The comparison bound R puts
  the calibration inputs within 1/1.1 of the range, so inputs up to 10 %
  beyond the calibration set still fall inside it;
* stage 1 is the odd polynomial of degree d_1 with the smallest maximum error
  against 1 on [eps, 1] (by oddness, against sign on both intervals);
* stage i + 1 is the odd polynomial of degree d_(i+1) with the smallest
  maximum error against 1 on the image of stage i's interval, which is
  [1 - tau_i, 1 + tau_i] for the stage's error tau_i;
* PolyComp(a, 0) = (1 + composite(a)) / 2.

Each stage is found by the Remez exchange on its interval (in the basis of
odd Chebyshev polynomials of the interval's right end, for conditioning) and
returned as odd monomial coefficients c with p(u) = sum_l c[l] u^(2l+1), the
form the encrypted evaluation takes.
"""
import numpy as np

A_DEFAULT = 1.0


def _basis(x, m, sc):
    t = np.asarray(x, dtype=np.float64) / sc
    return np.stack([np.polynomial.chebyshev.chebval(t, [0.0] * (2 * l + 1) + [1.0])
                     for l in range(m)], axis=-1)


def _extrema(err, n):
    """Indices of the largest |err| in each run of constant sign, n of them
    (the runs with the smallest extremum dropped from the ends); an exact
    zero joins the run before it."""
    sg = np.sign(err)
    for j in range(1, len(sg)):
        if sg[j] == 0:
            sg[j] = sg[j - 1]
    idx, start = [], 0
    for j in range(1, len(err) + 1):
        if j == len(err) or sg[j] != sg[start]:
            idx.append(start + int(np.argmax(np.abs(err[start:j]))))
            start = j
    while len(idx) > n:
        if abs(err[idx[0]]) < abs(err[idx[-1]]):
            idx.pop(0)
        else:
            idx.pop()
    return idx


def odd_minimax(lo, hi, degree, grid=40001, max_iter=100):
    """Odd polynomial of `degree` with the least max |p(x) - 1| on [lo, hi],
    0 < lo < hi. Returns (monomial coefficients c, max error, reference
    points, signed errors at the reference points)."""
    if degree % 2 != 1 or not 0 < lo < hi:
        raise ValueError("odd degree and 0 < lo < hi required")
    m = (degree + 1) // 2  # unknown coefficients
    n = m + 1  # reference points
    xs = np.linspace(lo, hi, grid)
    Bx = _basis(xs, m, hi)
    ref = lo + (hi - lo) * (1.0 - np.cos(np.pi * np.arange(n) / (n - 1))) / 2.0
    sol = None
    for _ in range(max_iter):
        M = np.concatenate([_basis(ref, m, hi), ((-1.0) ** np.arange(n))[:, None]], axis=1)
        sol = np.linalg.solve(M, np.ones(n))
        err = Bx @ sol[:m] - 1.0
        idx = _extrema(err, n)
        if len(idx) < n:
            break
        new = xs[idx]
        if np.allclose(new, ref, rtol=0, atol=(hi - lo) * 1e-12):
            break
        ref = new
    cheb = np.zeros(2 * m)
    cheb[1::2] = sol[:m]
    mono = np.polynomial.chebyshev.cheb2poly(cheb) * (1.0 / hi) ** np.arange(2 * m)
    c = [float(v) for v in mono[1::2]]
    lo_v, hi_v = image(c, lo, hi)
    ref_err = _basis(ref, m, hi) @ sol[:m] - 1.0
    return c, max(1.0 - lo_v, hi_v - 1.0), ref, ref_err


def eval_odd(u, c):
    u = np.asarray(u, dtype=np.float64)
    return sum(cl * u ** (2 * l + 1) for l, cl in enumerate(c))


def image(c, lo, hi):
    """[min, max] of the odd polynomial c over [lo, hi]: its values at the
    ends and at the real roots of its derivative inside."""
    d = np.zeros(2 * len(c))
    for l, cl in enumerate(c):
        d[2 * l] = (2 * l + 1) * cl  # coefficient of x^(2l) in p'
    r = np.roots(d[::-1]) if len(c) > 1 else np.array([])
    crit = [x.real for x in r if abs(x.imag) < 1e-9 * max(1.0, abs(x)) and lo < x.real < hi]
    v = eval_odd(np.array([lo, hi] + crit), c)
    return float(v.min()), float(v.max())


def composite(eps, degrees, A=A_DEFAULT):
    """Stages (lists of odd monomial coefficients) and the propagated error
    tau after each stage (the composite lies in [1 - tau, 1 + tau] on
    [eps, A])."""
    stages, taus = [], []
    lo, hi = eps, A
    for d in degrees:
        c, _, _, _ = odd_minimax(lo, hi, d)
        stages.append(c)
        lo, hi = image(c, lo, hi)  # the next stage's interval
        taus.append(max(1.0 - lo, hi - 1.0))
    return stages, taus
