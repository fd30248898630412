"""Pins for the oracle's KAN pieces (CPU only): Cox-de Boor (Eqs. 2-3)
against scipy's B-spline and the cubic knot values, Algorithm 2's index
algebra with exact comparisons, the f_n closed forms, Algorithm 3,
Eq. 13, the SiLU fit (Eqs. 11-12) against numpy's weighted Chebyshev fit,
the BSGS diagonal algebra by brute force, and the encrypted layer against
the HE-friendly FP64 KAN."""
import math

import numpy as np
import pytest

from oracle import calibrate, ckks, kan_he, kan_plain, silu_fit
from paper_2409_07751_gb300 import workloads as W


def _layer(G=5, k=3, n_in=3, n_out=2, seed=0):
    return W.make_model("t", seed=seed, widths=[n_in, n_out], G=G, k=k)[0]


def test_cox_de_boor_matches_scipy():
    si = pytest.importorskip("scipy.interpolate")
    for G, k in [(5, 3), (3, 2), (10, 5), (4, 1)]:
        L = _layer(G, k)
        t = kan_plain.knots(L)
        x = np.linspace(-1.0, 0.999, 101)
        B = kan_plain.bspline_exact(x, t, k)
        for m in range(G + k):
            ref = si.BSpline.basis_element(t[m:m + k + 2], extrapolate=False)(x)
            ref = np.nan_to_num(ref)
            assert np.abs(B[:, m] - ref).max() < 1e-12


def test_cubic_knot_values_and_partition_of_unity():
    L = _layer(5, 3)
    t = kan_plain.knots(L)
    B = kan_plain.bspline_exact(t[1:4], t, 3)
    # B_{0,3} at t_1, t_2, t_3 = 1/6, 2/3, 1/6
    assert np.allclose(B[:, 0], [1 / 6, 2 / 3, 1 / 6], atol=1e-15)
    x = np.linspace(-1, 0.99999, 1000)
    assert np.abs(kan_plain.bspline_exact(x, t, 3).sum(-1) - 1).max() < 1e-14
    # zero outside the extended grid
    assert np.abs(kan_plain.bspline_exact(np.array([t[-1] + 0.1, t[0] - 0.1]), t, 3)).max() == 0


def test_alg2_with_exact_comparison_is_cox_de_boor(monkeypatch):
    """Algorithm 2 with PolyComp replaced by the exact step reproduces Eq. 3."""
    monkeypatch.setattr(kan_plain, "polycomp0", lambda a, stages: (a > 0).astype(float))
    for G, k in [(5, 3), (10, 5), (3, 2)]:
        L = _layer(G, k)
        t = kan_plain.knots(L)
        x = np.random.default_rng(1).uniform(-1, 1, 300)
        assert np.abs(kan_plain.bspline_hef(x, t, k, 2.0, [3]) - kan_plain.bspline_exact(x, t, k)).max() < 1e-13


def test_b0_difference_form_with_exact_comparison_is_cox_de_boor(monkeypatch):
    """The difference form B_{m,0} = s_m - s_{m+1} of the order-0 basis,
    with PolyComp replaced by the exact step, also reproduces Eq. 3."""
    monkeypatch.setattr(kan_plain, "polycomp0", lambda a, stages: (a > 0).astype(float))
    for G, k in [(5, 3), (10, 5), (3, 2), (4, 0)]:
        L = _layer(G, k)
        t = kan_plain.knots(L)
        x = np.random.default_rng(2).uniform(-1, 1, 300)
        B = kan_plain.bspline_hef(x, t, k, 2.0, [3], b0="difference")
        assert np.abs(B - kan_plain.bspline_exact(x, t, k)).max() < 1e-13


def test_polycomp_odd_symmetry():
    """PolyComp(-a) = 1 - PolyComp(a) for the odd composites, the identity
    under which the product and difference forms of B_{m,0} coincide for
    exact steps."""
    a = np.random.default_rng(3).uniform(-1, 1, 1000)
    for stages in ([1], [3], [3, 3], [2, 5]):
        assert np.abs(kan_plain.polycomp0(-a, stages) - (1.0 - kan_plain.polycomp0(a, stages))).max() < 1e-15


def test_fn_closed_forms():
    assert kan_plain.fn_coeffs(1) == [1.5, -0.5]
    assert kan_plain.fn_coeffs(2) == [15 / 8, -10 / 8, 3 / 8]
    assert kan_plain.fn_coeffs(3) == [35 / 16, -35 / 16, 21 / 16, -5 / 16]
    for n in (1, 2, 3, 4):
        c = kan_plain.fn_coeffs(n)
        p = np.polynomial.Polynomial([0] + sum([[cl, 0] for cl in c], [])[:-1])
        assert abs(p(1.0) - 1) < 1e-15 and abs(p(-1.0) + 1) < 1e-15
        assert abs(p.deriv()(1.0)) < 1e-12
    s = kan_plain.polycomp0(np.array([-0.9, -0.3, 0.3, 0.9]), [3, 3, 3])
    assert np.allclose(s, [0, 0, 1, 1], atol=1e-3)


@pytest.mark.parametrize("name,data", [("kan_2_5_1", "uniform"), ("kan_4_8_4_1", "uniform"),
                                       ("kan_784_64_10", "blobs")])
def test_comparison_bound_keeps_polycomp_inputs_in_range(name, data):
    """Algorithm 2 feeds (x_rep - g1)/(2R) and (g2 - x_rep)/(2R) to PolyComp,
    which is accurate only on [-1, 1] (B-spline approximation section: inputs
    are scaled into [-1, 1] with R chosen from the data, larger than needed).
    Over the calibration set, every input x of every layer compared with
    every knot t_m gives |x - t_m| / (2R) <= 1/1.1 (the reading's 10 % margin),
    and the bound is attained: R is no larger than that margin requires."""
    model = W.make_model(name)
    n_in = model[0]["n_in"]
    X = W.uniform_inputs(256, n_in) if data == "uniform" else W.blob_images(64)
    m = calibrate.calibrate(model, X, 15, [3])
    _, acts = kan_plain.forward(m, X, "poly", "poly", collect=True)
    for L, a in zip(m, acts):
        t = kan_plain.knots(L)
        u = np.abs(a[..., None] - t) / (2.0 * L["R"])
        assert u.max() <= (1.0 / 1.1) * (1.0 + 1e-14)
        assert u.max() >= (1.0 / 1.1) * (1.0 - 1e-12)


def test_alg3_permutation_and_eq13():
    n_r, n_c = 4, 6
    P = kan_he.permutation_matrix(n_r, n_c)
    assert (P.sum(0) == 1).all() and (P.sum(1) == 1).all()
    L = _layer(3, 3, n_in=n_r, n_out=3)
    Bm = np.random.default_rng(2).normal(size=(n_r, n_c))  # B[i, m]
    row_major = Bm.reshape(-1)                              # i*(g+k) + m
    col_tile = Bm.T.reshape(-1)                              # m*n_i + i
    assert np.allclose(P @ col_tile, row_major)
    Wp, Wf = kan_he.lazy_weights(L), kan_he.fused_weights(L)
    assert np.allclose(Wf @ col_tile, Wp @ row_major, atol=1e-14)
    # and W' row-major is the einsum of the per-edge spline
    y = np.einsum("im,oim,oi->o", Bm, L["coef"], L["w_s"])
    assert np.allclose(Wp @ row_major, y)


def test_coltile():
    Gm = np.arange(12.0).reshape(3, 4)
    assert list(kan_he.coltile(Gm, 2, 4)) == [1, 5, 9, 2, 6, 10]


def test_silu_fit_matches_numpy_weighted_chebfit():
    lo, hi, mu, sig = -6.0, 5.0, -0.3, 1.4
    a = silu_fit.fit_silu(lo, hi, mu, sig, 12, 4000)
    x = np.linspace(lo, hi, 4000)
    y = (2 * x - (lo + hi)) / (hi - lo)
    w = np.where(np.abs(x - mu) <= 3 * sig, 10.0, 1.0)
    ref = np.polynomial.chebyshev.chebfit(y, kan_plain.silu(x), 12, w=np.sqrt(w))
    assert np.abs(a - ref).max() < 1e-9
    # weighted normal equations: V^T W r = 0
    V = np.polynomial.chebyshev.chebvander(y, 12)
    r = kan_plain.silu(x) - V @ a
    assert np.abs(V.T @ (w * r)).max() < 1e-8
    assert silu_fit.silu_range(0.0, 1.0, -3.0, 7.0) == (-3.0, 5.0)
    assert silu_fit.silu_range(0.0, 1.0, -9.0, 2.0) == (-5.0, 2.0)


def test_bsgs_diagonal_algebra_bruteforce():
    S = 64
    rng = np.random.default_rng(3)
    for n_out, n in [(3, 20), (8, 8), (5, 32), (2, 3), (16, 64)]:
        M = rng.normal(size=(n_out, n))
        plan = kan_he.bsgs_plan(n_out, n, S)
        D = kan_he.diagonals(M, plan, S)
        v = np.zeros(S)
        v[:n] = rng.normal(size=n)
        npad = plan["npad"]
        if npad < S:
            v = v + np.roll(v, npad)  # rot(v, -npad)
        rot = lambda a, t: np.roll(a, -t)
        z = np.zeros(S)
        for i in range(plan["g2"]):
            inner = sum(np.roll(D[plan["g1"] * i + j], plan["g1"] * i) * rot(v, j) for j in range(plan["g1"]))
            z += rot(inner, plan["g1"] * i)
        for s in plan["folds"]:
            z = z + rot(z, s)
        assert np.allclose(z[:n_out], M @ v[:n])


@pytest.fixture(scope="module")
def he_small():
    ctx = ckks.Ctx(ckks.Params(log_n=7, n_scale=17, n_special=2))
    return ctx


def test_alg1_repeat_packing(he_small):
    ctx = he_small
    n_i, G, k = 3, 5, 3
    J = math.ceil(math.log2(G + 2 * k))
    keys = ckks.Keys(ctx, 1, rot_steps=[-n_i * 2 ** (j - 1) for j in range(1, J + 1)])
    x = np.zeros(ctx.slots)
    x[:n_i] = [0.1, -0.2, 0.3]
    x[n_i:] = 5.0  # garbage outside the input slots must be masked away
    c = ckks.encrypt(ctx, keys, x, ctx.L, 2)
    xr = ckks.mul_plain(ctx, c, np.ones(n_i))
    for j in range(1, J + 1):
        xr = ckks.add(ctx, xr, ckks.rotate(ctx, keys, xr, -n_i * 2 ** (j - 1)))
    d = ckks.decrypt(ctx, keys, xr)
    ref = np.zeros(ctx.slots)
    ref[: n_i * 2 ** J] = np.tile(x[:n_i], 2 ** J)
    assert np.abs(d - ref).max() < 1e-6


def test_he_polynomials(he_small):
    ctx = he_small
    keys = ckks.Keys(ctx, 2)
    rng = np.random.default_rng(4)
    y = rng.uniform(-1, 1, ctx.slots)
    c = ckks.encrypt(ctx, keys, y, ctx.L, 2)
    for d in (3, 7, 15, 27):
        a = rng.normal(size=d + 1) / (1 + np.arange(d + 1))
        out = kan_he.eval_cheb(ctx, keys, c, a)
        assert np.abs(ckks.decrypt(ctx, keys, out) - np.polynomial.chebyshev.chebval(y, a)).max() < 1e-5
        assert ctx.L - out.level <= math.ceil(math.log2(d + 1)) + 1
    for stages in ([1], [3], [3, 1]):
        out = kan_he.polycomp0(ctx, keys, c, stages)
        assert np.abs(ckks.decrypt(ctx, keys, out) - kan_plain.polycomp0(y, stages)).max() < 1e-5


def test_he_odd_polynomial_split_evaluation(he_small, monkeypatch):
    """eval_odd equals sum_l c_l y^(2l+1) for 1..8 coefficients (zeros
    included), at depth ceil(log2(degree + 1)), with 5 ciphertext products
    for f_3 (degree 7: u^2, u^4 and one per split)."""
    ctx = he_small
    keys = ckks.Keys(ctx, 2)
    rng = np.random.default_rng(6)
    y = rng.uniform(-1, 1, ctx.slots)
    c = ckks.encrypt(ctx, keys, y, ctx.L, 2)
    for n in range(1, 9):
        cf = list(rng.normal(size=n))
        if n >= 3:
            cf[1] = 0.0
        out = kan_he.eval_odd(ctx, keys, c, cf, 0.25)
        ref = 0.25 + sum(cl * y ** (2 * l + 1) for l, cl in enumerate(cf))
        assert np.abs(ckks.decrypt(ctx, keys, out) - ref).max() < 1e-5, n
        assert ctx.L - out.level == math.ceil(math.log2(2 * n)), n
    calls = []
    real = ckks.mul
    monkeypatch.setattr(ckks, "mul", lambda *a: calls.append(1) or real(*a))
    kan_he.eval_odd(ctx, keys, c, kan_plain.fn_coeffs(3))
    assert len(calls) == 5


def test_he_bsgs_matvec(he_small):
    ctx = he_small
    rng = np.random.default_rng(5)
    n_out, n = 5, 20
    M = rng.normal(size=(n_out, n))
    plan = kan_he.bsgs_plan(n_out, n, ctx.slots)
    steps = [-plan["npad"]] + list(range(1, plan["g1"])) + [plan["g1"] * i for i in range(1, plan["g2"])] + plan["folds"]
    keys = ckks.Keys(ctx, 3, rot_steps=steps)
    v = np.zeros(ctx.slots)
    v[:n] = rng.uniform(-1, 1, n)
    c = ckks.encrypt(ctx, keys, v, ctx.L, 2)
    c = ckks.add(ctx, c, ckks.rotate(ctx, keys, c, -plan["npad"]))
    out = kan_he.bsgs_matvec(ctx, keys, c, M, plan)
    assert np.abs(ckks.decrypt(ctx, keys, out, n_out) - M @ v[:n]).max() < 1e-6


@pytest.mark.parametrize("n_out,n", [(5, 20), (16, 40), (2, 64)])
def test_he_bsgs_matvec_double_hoisted(he_small, n_out, n):
    """Double hoisting (baby steps kept in QP_l, one division by P q_l per
    giant step): decrypts to the dense M v in FP64, like the hoisted form
    (the two differ only in the rounding of their divisions), one level."""
    ctx = he_small
    rng = np.random.default_rng(5 + n)
    M = rng.normal(size=(n_out, n))
    plan = kan_he.bsgs_plan(n_out, n, ctx.slots)
    steps = [-plan["npad"]] + list(range(1, plan["g1"])) + [plan["g1"] * i for i in range(1, plan["g2"])] + plan["folds"]
    keys = ckks.Keys(ctx, 3, rot_steps=steps)
    v = np.zeros(ctx.slots)
    v[:n] = rng.uniform(-1, 1, n)
    c = ckks.encrypt(ctx, keys, v, ctx.L, 2)
    if plan["npad"] < ctx.slots:
        c = ckks.add(ctx, c, ckks.rotate(ctx, keys, c, -plan["npad"]))
    dbl = kan_he.bsgs_matvec_double(ctx, keys, c, M, plan)
    one = kan_he.bsgs_matvec(ctx, keys, c, M, plan)
    assert dbl.level == one.level == ctx.L - 1 and dbl.scale == one.scale
    d = ckks.decrypt(ctx, keys, dbl, n_out)
    assert np.abs(d - M @ v[:n]).max() < 1e-6
    assert np.abs(d - ckks.decrypt(ctx, keys, one, n_out)).max() < 1e-6
    assert not np.array_equal(dbl.data, one.data)  # a different rounding, not the same words


def test_he_kan_double_hoisted_matches_hef(he_small):
    ctx = he_small
    model = [dict(L, bsgs="double") for L in W.make_model("t", widths=[3, 4, 2], G=3, k=2)]
    X = W.uniform_inputs(100, 3)
    m = calibrate.calibrate(model, X, 7, [1])
    keys = ckks.Keys(ctx, 1, rot_steps=kan_he.model_rotations(m, ctx.slots))
    c = ckks.encrypt(ctx, keys, X[0], ctx.L, 2, 0)
    out = kan_he.infer(ctx, keys, c, m)
    hef = kan_plain.forward(m, X[:1], "poly", "poly")[0]
    assert np.abs(ckks.decrypt(ctx, keys, out, 2) - hef).max() < 1e-5


def test_he_kan_matches_hef(he_small):
    ctx = he_small
    model = W.make_model("t", widths=[3, 4, 2], G=3, k=2)
    X = W.uniform_inputs(100, 3)
    m = calibrate.calibrate(model, X, 7, [1])
    keys = ckks.Keys(ctx, 1, rot_steps=kan_he.model_rotations(m, ctx.slots))
    for b in range(2):
        c = ckks.encrypt(ctx, keys, X[b], ctx.L, 2, b)
        out = kan_he.infer(ctx, keys, c, m)
        dec = ckks.decrypt(ctx, keys, out, 2)
        hef = kan_plain.forward(m, X[b:b + 1], "poly", "poly")[0]
        assert np.abs(dec - hef).max() < 1e-5


@pytest.mark.parametrize("G_,k_", [(3, 2), (4, 0)])
def test_he_kan_b0_difference_form_matches_hef(he_small, G_, k_):
    """With B_{m,0} = s_m - s_{m+1} (one comparison per knot, rot(s, n_i)
    for s_{m+1}, no product) the encrypted network equals the HE-friendly
    KAN of the same form and, where the spline branch is the deeper one
    (k >= 1 here), ends one level higher per layer than the product form."""
    ctx = he_small
    model = W.make_model("t", widths=[3, 4, 2], G=G_, k=k_)
    for L in model:
        L["b0"] = "difference"
    X = W.uniform_inputs(100, 3)
    m = calibrate.calibrate(model, X, 7, [1])
    keys = ckks.Keys(ctx, 1, rot_steps=kan_he.model_rotations(m, ctx.slots))
    c = ckks.encrypt(ctx, keys, X[0], ctx.L, 2, 0)
    out = kan_he.infer(ctx, keys, c, m)
    dec = ckks.decrypt(ctx, keys, out, 2)
    hef = kan_plain.forward(m, X[:1], "poly", "poly")[0]
    assert np.abs(dec - hef).max() < 1e-5
    mp = [dict(L, b0="product") for L in m]
    keys_p = ckks.Keys(ctx, 1, rot_steps=kan_he.model_rotations(mp, ctx.slots))
    out_p = kan_he.infer(ctx, keys_p, ckks.encrypt(ctx, keys_p, X[0], ctx.L, 2, 0), mp)
    assert out.level - out_p.level == (len(m) if k_ >= 1 else 0)


@pytest.mark.parametrize("G_,k_", [(1, 0), (4, 0), (2, 1)])
def test_he_kan_degenerate_grids_match_hef(he_small, G_, k_):
    """Order-0 splines and a single interval: the encrypted layer still
    equals the HE-friendly KAN (for k = 0 the basis must be zero outside its
    n_i g slots before the matvec replicates it)."""
    ctx = he_small
    model = W.make_model("t", widths=[3, 2], G=G_, k=k_)
    X = W.uniform_inputs(64, 3)
    m = calibrate.calibrate(model, X, 5, [1])
    keys = ckks.Keys(ctx, 1, rot_steps=kan_he.model_rotations(m, ctx.slots))
    c = ckks.encrypt(ctx, keys, X[0], ctx.L, 2, 0)
    out = kan_he.infer(ctx, keys, c, m)
    dec = ckks.decrypt(ctx, keys, out, 2)
    hef = kan_plain.forward(m, X[:1], "poly", "poly")[0]
    assert np.abs(dec - hef).max() < 1e-5


def test_he_naive_permutation_method_matches_hef(he_small):
    """The naive method (HE permutation by P of Algorithm 3, then W') gives
    the same network values as lazy combination, one level deeper."""
    ctx = he_small
    model = W.make_model("t", widths=[3, 4, 2], G=3, k=2)
    X = W.uniform_inputs(100, 3)
    m = calibrate.calibrate(model, X, 7, [1])
    naive = [dict(L, naive=True) for L in m]
    keys = ckks.Keys(ctx, 1, rot_steps=kan_he.model_rotations(naive, ctx.slots))
    c = ckks.encrypt(ctx, keys, X[0], ctx.L, 2, 0)
    lazy = kan_he.layer_eval(ctx, keys, c, m[0])
    out = kan_he.layer_eval(ctx, keys, c, naive[0])
    assert out.level == lazy.level - 1
    full = kan_he.infer(ctx, keys, c, naive)
    hef = kan_plain.forward(m, X[:1], "poly", "poly")[0]
    assert np.abs(ckks.decrypt(ctx, keys, full, 2) - hef).max() < 1e-5


def test_permutation_bsgs_reorders_coltile_to_row_major():
    """The naive method's P matvec on the BSGS diagonal algebra (plaintext
    slots): ColTile order m n_i + i in, row-major i (g+k) + m out."""
    S, n_i, nb = 256, 5, 6
    n = n_i * nb
    P = kan_he.permutation_matrix(n_i, nb)
    plan = kan_he.bsgs_plan(n, n, S)
    D = kan_he.diagonals(P, plan, S)
    rng = np.random.default_rng(8)
    B = rng.normal(size=(n_i, nb))  # B[i, m]
    v = np.zeros(S)
    v[:n] = B.T.reshape(-1)  # ColTile
    v = v + np.roll(v, plan["npad"])  # replicate to [0, 2 npad)

    def rot(a, t):
        return np.roll(a, -t)

    z = np.zeros(S)
    for i in range(plan["g2"]):
        inner = sum(np.roll(D[plan["g1"] * i + j], plan["g1"] * i) * rot(v, j) for j in range(plan["g1"]))
        z += rot(inner, plan["g1"] * i)
    assert np.allclose(z[:n], B.reshape(-1))
    assert np.allclose(z[n:], 0.0)


def test_remez_closed_forms_and_equioscillation():
    """Remez pins: the minimax cubic of x^4 on [-1, 1] is x^4 - T_4/8 and the
    minimax quadratic of |x| is x^2 + 1/8 (Chebyshev alternation); the SiLU
    minimax error equioscillates at d + 2 points."""
    c = silu_fit.fit_silu(-1, 1, 0, 1, 3, 20001, "remez", f=lambda x: x ** 4)
    assert np.abs(c - [3 / 8, 0, 1 / 2, 0]).max() < 1e-9
    c = silu_fit.fit_silu(-1, 1, 0, 1, 2, 20001, "remez", f=np.abs)
    assert np.abs(c - [5 / 8, 0, 1 / 2]).max() < 1e-6
    lo, hi, d = -12.4, 14.74, 10
    c = silu_fit.fit_silu(lo, hi, 0, 1, d, 10000, "remez")
    x = np.linspace(lo, hi, 10000)
    e = kan_plain.silu(x) - np.polynomial.chebyshev.chebval((2 * x - (lo + hi)) / (hi - lo), c)
    ext = [a + int(np.argmax(np.abs(e[a:b]))) for a, b in silu_fit._runs(e)]
    assert len(ext) >= d + 2
    mags = np.abs(e[ext])
    assert mags.max() - np.sort(mags)[-(d + 2)] < 1e-6 * mags.max()


def test_ols_matches_numpy_chebfit():
    lo, hi = -9.77, 11.01
    a = silu_fit.fit_silu(lo, hi, 0.0, 1.0, 10, 3000, "ols")
    x = np.linspace(lo, hi, 3000)
    ref = np.polynomial.chebyshev.chebfit((2 * x - (lo + hi)) / (hi - lo), kan_plain.silu(x), 10)
    assert np.abs(a - ref).max() < 1e-9
