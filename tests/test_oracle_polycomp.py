"""Pins for the oracle's composite minimax comparison (PolyComp of
Algorithm 2 by minimax composites, Lee et al. 2021), CPU only.

Each stage is checked against something other than its own Remez loop: the
degree-1 closed form, a linear program over a dense grid (an independent way
to the same best approximation), the alternation theorem (a best
approximation equioscillates), and the composite's error bound evaluated on a
dense FP64 grid; the encrypted evaluation is checked against the plaintext
composite."""
import numpy as np
import pytest

from oracle import ckks, kan_he, kan_plain, polycomp


def test_degree_one_closed_form():
    # the best c x against 1 on [lo, hi] equalises the errors at both ends:
    # c = 2 / (lo + hi), error (hi - lo) / (hi + lo)
    for lo, hi in ((0.1, 1 / 1.1), (0.5, 1.5), (0.02, 0.9)):
        c, err, _, _ = polycomp.odd_minimax(lo, hi, 1)
        assert c[0] == pytest.approx(2.0 / (lo + hi), rel=1e-12)
        assert err == pytest.approx((hi - lo) / (hi + lo), rel=1e-9)


@pytest.mark.parametrize("lo,hi,deg", [(0.1, 1 / 1.1, 7), (0.05, 1 / 1.1, 7), (0.5, 1.5, 15),
                                       (0.9, 1.1, 7), (0.2, 1 / 1.1, 15)])
def test_matches_linear_program(lo, hi, deg):
    """min E s.t. |p(x_j) - 1| <= E on 4001 grid points, solved by scipy's
    LP (HiGHS) over odd Chebyshev coefficients: the same error and the same
    polynomial to the grid's resolution."""
    linprog = pytest.importorskip("scipy.optimize").linprog
    m = (deg + 1) // 2
    xs = np.linspace(lo, hi, 4001)
    B = np.stack([np.polynomial.chebyshev.chebval(xs / hi, [0] * (2 * l + 1) + [1])
                  for l in range(m)], axis=1)
    # variables: m coefficients, then E; minimise E
    cost = np.zeros(m + 1)
    cost[-1] = 1.0
    ones = np.ones((len(xs), 1))
    A_ub = np.vstack([np.hstack([B, -ones]), np.hstack([-B, -ones])])
    b_ub = np.concatenate([np.ones(len(xs)), -np.ones(len(xs))])
    res = linprog(cost, A_ub=A_ub, b_ub=b_ub, bounds=[(None, None)] * (m + 1), method="highs")
    assert res.status == 0
    E_lp = res.x[-1]
    c, err, _, _ = polycomp.odd_minimax(lo, hi, deg)
    assert err == pytest.approx(E_lp, rel=2e-3, abs=1e-12)
    p_lp = B @ res.x[:m]
    p_rz = polycomp.eval_odd(xs, c)
    assert np.abs(p_lp - p_rz).max() <= 0.05 * err + 1e-12


@pytest.mark.parametrize("lo,hi,deg", [(0.1, 1 / 1.1, 7), (0.3, 1 / 1.1, 15), (0.6, 1.4, 15)])
def test_equioscillation(lo, hi, deg):
    """(deg + 3) / 2 reference points with alternating errors of equal size,
    equal to the maximum error over the interval (alternation theorem)."""
    c, err, ref, ref_err = polycomp.odd_minimax(lo, hi, deg)
    n = (deg + 1) // 2 + 1
    assert len(ref) == n and np.all(np.diff(ref) > 0)
    assert np.all(np.sign(ref_err[1:]) == -np.sign(ref_err[:-1]))
    assert np.abs(ref_err).max() == pytest.approx(np.abs(ref_err).min(), rel=1e-6)
    assert np.abs(ref_err).max() == pytest.approx(err, rel=1e-6)


@pytest.mark.parametrize("eps,degs", [(0.1, (7, 15)), (0.02, (7, 7, 7, 7)), (0.02, (7, 15, 15))])
def test_composite_bound_on_dense_grid(eps, degs):
    """On 10^6 points of [eps, A] the composite stays within the propagated
    error; it is odd; and on the whole of [-A, A] (the transition included)
    it stays within that bound of [-1, 1], so no input blows up."""
    A = polycomp.A_DEFAULT
    stages, taus = polycomp.composite(eps, degs)
    assert all(t < 1 for t in taus)
    x = np.linspace(eps, A, 1_000_001)
    u = x
    for c in stages:
        u = polycomp.eval_odd(u, c)
    # (to the FP64 rounding of evaluating the stages, ~1e-13)
    assert np.abs(u - 1.0).max() <= taus[-1] * (1 + 1e-9) + 1e-13
    v = -x
    for c in stages:
        v = polycomp.eval_odd(v, c)
    assert np.abs(v + u).max() < 1e-12  # odd up to FP64 rounding
    y = np.linspace(-A, A, 400_001)
    for c in stages:
        y = polycomp.eval_odd(y, c)
    assert np.abs(y).max() <= 1.0 + taus[-1] + 1e-12
    # PolyComp(a, 0) = (1 + f(a)) / 2 through the plaintext KAN's path
    assert np.array_equal(kan_plain.polycomp0(x, stages), 0.5 + 0.5 * u)


def test_he_minimax_polycomp_matches_plaintext():
    """The encrypted composite (odd split evaluation, oracle CKKS at N = 2^6)
    decrypts to the plaintext composite within CKKS noise."""
    stages, _ = polycomp.composite(0.1, (7, 15))
    ctx = ckks.Ctx(ckks.Params(log_n=6, n_scale=10, n_special=2))
    keys = ckks.Keys(ctx, 3)
    a = np.linspace(-1 / 1.1, 1 / 1.1, ctx.slots)
    ct = ckks.encrypt(ctx, keys, a, ctx.L, 5)
    out = kan_he.polycomp0(ctx, keys, ct, stages)
    assert ctx.L - out.level == 3 + 4 + 0  # depth ceil(log2(4)) + 1 + ceil(log2(8)) + 1
    dec = ckks.decrypt(ctx, keys, out)
    assert np.abs(dec - kan_plain.polycomp0(a, stages)).max() < 1e-4
