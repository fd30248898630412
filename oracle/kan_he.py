"""Encrypted KAN layer on the oracle CKKS (test infrastructure only).

Follows the paper's Method section step by step:

* Algorithm 1 (fast repeat packing): mask x to its n_i slots, then
  ceil(log2(g+2k)) times add the ciphertext rotated right by n_i 2^(j-1).
  Reading: the 1/(2R) input scaling of Algorithm 2 (line 4) is folded into
  the mask, so the comparison inputs need no extra level.
* Algorithm 2 (B-spline basis): ColTile'd knot vectors, PolyComp via a
  composite of odd polynomials (minimax stages as in Lee et al., built by
  polycomp.py, or Cheon et al.'s closed-form f_n) with its last stage
  returning (1 + f)/2, B0 = x1 (x) x2, then k recursion steps
  b <- A1 (x_rep - t1) (x) b + A2 (t3 - x_rep) (x) rot(b, n_i). Reading: the two
  products of a step share one relinearisation; A1, A2 are zero outside the
  valid ColTile blocks.
* Lazy combination and Algorithm 3: W_f = W' P (Eq. 13) with
  W'[o, i(g+k) + m] = w_s[o, i] c[o, i, m].
* SiLU (Eqs. 11-12): the fitted Chebyshev polynomial evaluated by a
  Paterson-Stockmeyer-style baby-step / giant-step recursion.
* Linear layers: baby-step giant-step diagonal matvec (Halevi-Shoup) with
  hoisted baby-step rotations.
"""
import math

import numpy as np

from . import ckks
from .kan_plain import knots, stage_coeffs


def pow2ceil(n):
    return 1 << max(0, (int(n) - 1).bit_length())


def rep_bits(layer):
    """J of Algorithm 1: 2^J >= the ColTile blocks Algorithm 2 compares,
    g + 2k (one per order-0 basis function), or g + 2k + 1 for the
    difference form of B_{m,0}, which compares against every knot."""
    blocks = layer["G"] + 2 * layer["k"] + (1 if layer.get("b0") == "difference" else 0)
    return math.ceil(math.log2(blocks))


# ------------------------------------------------------------------ Algorithm 3
def permutation_matrix(n_r, n_c):
    """Algorithm 3 (1-indexed in the paper): P[(r-1)n_c + c][(c-1)n_r + r] = 1."""
    P = np.zeros((n_r * n_c, n_r * n_c))
    for r in range(1, n_r + 1):
        for c in range(1, n_c + 1):
            j_c = (c - 1) * n_r + r
            j_r = (r - 1) * n_c + c
            P[j_r - 1, j_c - 1] = 1.0
    return P


def lazy_weights(layer):
    """W' (n_o x n_i(g+k)), row-major basis index i(g+k) + m."""
    n_o, n_i = layer["n_out"], layer["n_in"]
    nb = layer["G"] + layer["k"]
    Wp = (layer["w_s"][:, :, None] * layer["coef"]).reshape(n_o, n_i * nb)
    return Wp


def fused_weights(layer):
    """Eq. 13: W_f = W' P (columns in ColTile order m n_i + i)."""
    return lazy_weights(layer) @ permutation_matrix(layer["n_in"], layer["G"] + layer["k"])


# ------------------------------------------------------------------ ColTile
def coltile(Gm, l, r):
    """ColTile(G, l, r): columns l..r-1 (1-indexed) of G concatenated column-major."""
    return np.concatenate([Gm[:, c - 1] for c in range(l, r)]) if r > l else np.zeros(0)


def grid_matrix(layer):
    t = knots(layer)
    return np.tile(t[None, :], (layer["n_in"], 1))


# ------------------------------------------------------------------ BSGS plan
def bsgs_plan(n_out, n, slots):
    no = pow2ceil(n_out)
    npad = pow2ceil(max(n, no))
    if npad > slots:
        raise ValueError("matrix does not fit the slots")
    g1 = 1 << ((no.bit_length() - 1 + 1) // 2)
    g2 = no // g1
    folds = []
    s = npad // 2
    while s >= no:
        folds.append(s)
        s //= 2
    return dict(no=no, npad=npad, g1=g1, g2=g2, folds=folds)


def diagonals(M, plan, slots):
    """d_t[s] = M[s mod no][(s+t) mod npad] for s < npad (zero where undefined)."""
    n_out, n = M.shape
    no, npad = plan["no"], plan["npad"]
    Mp = np.zeros((no, npad))
    Mp[:n_out, :n] = M
    s = np.arange(npad)
    D = np.zeros((no, slots))
    for t in range(no):
        D[t, :npad] = Mp[s % no, (s + t) % npad]
    return D


def bsgs_matvec(ctx, keys, v, M, plan):
    """y[0:n_out] = M v; v must read v[(s+t) mod npad] at slot s+t for s < npad."""
    S = ctx.slots
    D = diagonals(M, plan, S)
    g1, g2 = plan["g1"], plan["g2"]
    baby = ckks.rotate_many(ctx, keys, v, list(range(g1)))
    lv = v.level
    z = None
    for i in range(g2):
        acc = None
        Spt = ckks.plain_scale(ctx, v.scale, lv)
        for j in range(g1):
            d = np.roll(D[g1 * i + j], g1 * i)  # rot(d, -g1 i)
            pt = ckks.encode(ctx, d, lv, Spt)
            prod = np.zeros_like(v.data)
            ctx.L_.or_mul_plain(ctx.h, baby[j].data.ctypes.data, pt.ctypes.data, 2, lv + 1,
                                prod.ctypes.data)
            if acc is None:
                acc = prod
            else:
                o = np.zeros_like(acc)
                ctx.L_.or_add(ctx.h, acc.ctypes.data, prod.ctypes.data, 2, lv + 1, 0, o.ctypes.data)
                acc = o
        inner = ckks.rescale(ctx, ckks.Ct(acc, lv, v.scale * Spt))
        if i > 0:
            inner = ckks.rotate(ctx, keys, inner, g1 * i)
        z = inner if z is None else ckks.add(ctx, z, inner)
    for s in plan["folds"]:
        z = ckks.add(ctx, z, ckks.rotate(ctx, keys, z, s))
    return z


def bsgs_matvec_double(ctx, keys, v, M, plan):
    """bsgs_matvec with double hoisting (layer option bsgs = "double"): the
    baby-step rotations stay in QP_l (one ModUp, no ModDown), each giant
    step's diagonal products are summed over QP_l with the diagonals encoded
    over QP_l, and the sum is divided by P q_level once (ModDown and the
    rescale of the products in one rounded division), then rotated by g1 i."""
    S = ctx.slots
    D = diagonals(M, plan, S)
    g1, g2 = plan["g1"], plan["g2"]
    lv = v.level
    R = ckks.rotate_many_qp(ctx, keys, v, list(range(g1)))
    Spt = ckks.plain_scale(ctx, v.scale, lv)
    z = None
    for i in range(g2):
        acc = np.zeros_like(R[0])
        for j in range(g1):
            d = np.roll(D[g1 * i + j], g1 * i)  # rot(d, -g1 i)
            ckks.qp_mul_plain_acc(ctx, R[j], ckks.encode_qp(ctx, d, lv, Spt), lv, acc)
        inner = ckks.div_p_ql(ctx, acc, lv, v.scale * Spt)
        if i > 0:
            inner = ckks.rotate(ctx, keys, inner, g1 * i)
        z = inner if z is None else ckks.add(ctx, z, inner)
    for s in plan["folds"]:
        z = ckks.add(ctx, z, ckks.rotate(ctx, keys, z, s))
    return z


def matvec(ctx, keys, v, M, plan, layer):
    """The layer's BSGS form: hoisted (default) or double-hoisted."""
    if layer.get("bsgs", "single") == "double":
        return bsgs_matvec_double(ctx, keys, v, M, plan)
    return bsgs_matvec(ctx, keys, v, M, plan)


# ------------------------------------------------------------------ polynomials
def eval_odd(ctx, keys, u, c, const=0.0):
    """sum_l c[l] u^(2l+1) + const. The coefficient list is padded to 2^K
    and split in halves: p = A + u^(2^K) B with A, B the odd polynomials of
    the lower and upper halves, recursively; a single coefficient is c_l u
    (one constant product). Each level of the recursion costs one depth, so
    the result is at depth K + 1 = ceil(log2(deg + 1)); f_3 (degree 7) takes
    5 ciphertext products (u^2, u^4 and three splits). Reading: the paper
    fixes the comparison polynomial, not its evaluation order."""
    K = max(0, math.ceil(math.log2(len(c))))
    c = list(c) + [0.0] * ((1 << K) - len(c))
    pw = {1: u}
    for k in range(1, K + 1):  # u^(2^k)
        pw[1 << k] = ckks.mul(ctx, keys, pw[1 << (k - 1)], pw[1 << (k - 1)])

    def rec(lo, k):
        if k == 0:
            return ckks.mul_const(ctx, u, c[lo]) if c[lo] != 0.0 else None
        half = 1 << (k - 1)
        A = rec(lo, k - 1)
        B = rec(lo + half, k - 1)
        if B is None:
            return A
        P = ckks.mul(ctx, keys, B, pw[1 << k])
        if A is None:
            return P
        return ckks.add(ctx, ckks.level_down(ctx, A, P.level), P)

    out = rec(0, K)
    if const != 0.0:
        out = ckks.add_const(ctx, out, const)
    return out


def polycomp0(ctx, keys, a, stages):
    """PolyComp(a, 0) = (1 + f(a))/2 with f the composite of the stages
    (f_n by order n, or explicit odd coefficient lists), first stage first."""
    u = a
    for s, st in enumerate(stages):
        c = stage_coeffs(st)
        if s == len(stages) - 1:
            u = eval_odd(ctx, keys, u, [0.5 * x for x in c], 0.5)
        else:
            u = eval_odd(ctx, keys, u, c)
    return u


def eval_cheb(ctx, keys, y, a):
    """sum_j a_j T_j(y) by baby steps T_1..T_m (m a power of two with
    m >= sqrt(d+1)) and giant steps T_{m 2^i}, splitting
    p = q T_D + r with q_0 = a_D, q_i = 2 a_{D+i}, r_j = a_j - a_{2D-j}."""
    a = [float(x) for x in a]
    d = len(a) - 1
    m = pow2ceil(math.ceil(math.sqrt(d + 1)))
    T = {1: y}
    for i in range(2, m + 1):
        if i & (i - 1) == 0:
            sq = ckks.mul(ctx, keys, T[i // 2], T[i // 2])
            T[i] = ckks.add_const(ctx, ckks.mul_int(ctx, sq, 2), -1.0)
        else:
            hb = 1 << (i.bit_length() - 1)
            lo = i - hb
            pr = ckks.mul_int(ctx, ckks.mul(ctx, keys, T[hb], T[lo]), 2)
            if hb - lo == 0:
                T[i] = ckks.add_const(ctx, pr, -1.0)
            else:
                T[i] = ckks.sub(ctx, pr, ckks.level_down(ctx, T[hb - lo], pr.level))
    Gs = {m: T[m]}
    D = m
    while 2 * D <= d:
        sq = ckks.mul(ctx, keys, Gs[D], Gs[D])
        Gs[2 * D] = ckks.add_const(ctx, ckks.mul_int(ctx, sq, 2), -1.0)
        D *= 2

    def rec(c):
        deg = len(c) - 1
        if deg < m:
            if deg == 0:
                return c[0]
            return ckks.lincomb(ctx, [T[i] for i in range(1, deg + 1)], c[1:], c[0])
        D = m
        while 2 * D <= deg:
            D *= 2
        q = [c[D]] + [2.0 * c[D + i] for i in range(1, deg - D + 1)]
        r = list(c[:D])
        for i in range(1, deg - D + 1):
            r[D - i] -= c[D + i]
        Q = rec(q)
        R = rec(r)
        if isinstance(Q, float):
            P = ckks.lincomb(ctx, [Gs[D]], [Q])
        else:
            P = ckks.mul(ctx, keys, Q, Gs[D])
        if isinstance(R, float):
            return ckks.add_const(ctx, P, R)
        lv = min(P.level, R.level)
        return ckks.add(ctx, ckks.level_down(ctx, P, lv), ckks.level_down(ctx, R, lv))

    return rec(a)


# ------------------------------------------------------------------ layer
def layer_rotations(layer, slots):
    """Every rotation step the layer schedule uses."""
    K, n_c = chunking(layer, slots)
    n_o, G, k = layer["n_out"], layer["G"], layer["k"]
    n_i = n_c
    J = rep_bits(layer)
    steps = {-n_i * 2 ** (j - 1) for j in range(1, J + 1)}
    steps.add(n_i)
    plans = [(n_o, n_i * (G + k)), (n_o, n_i)]
    if layer.get("naive"):
        plans.append((n_i * (G + k), n_i * (G + k)))
    for n_out, n in plans:
        p = bsgs_plan(n_out, n, slots)
        if p["npad"] < slots:
            steps.add(-p["npad"])
        steps.update(range(1, p["g1"]))
        steps.update(p["g1"] * i for i in range(1, p["g2"]))
        steps.update(p["folds"])
    steps.discard(0)
    return sorted(steps)


def layer_eval(ctx, keys, x, layer):
    S = ctx.slots
    n_i, n_o, G, k = layer["n_in"], layer["n_out"], layer["G"], layer["k"]
    R = layer["R"]
    J = rep_bits(layer)
    if n_i * 2 ** J > S:
        raise ValueError("repeat packing needs n_i * 2^J <= N/2")
    mask = np.ones(n_i)

    # SiLU branch: y = affine(x) on the masked slots, replicated to period npad
    lo, hi = layer["silu_lo"], layer["silu_hi"]
    sa, sb = 2.0 / (hi - lo), -(hi + lo) / (hi - lo)
    y = ckks.add_plain(ctx, ckks.mul_plain(ctx, x, sa * mask), sb * mask)
    plan_b = bsgs_plan(n_o, n_i, S)
    if plan_b["npad"] < S:
        y = ckks.add(ctx, y, ckks.rotate(ctx, keys, y, -plan_b["npad"]))
    v = eval_cheb(ctx, keys, y, layer["silu_cheb"])
    yb = matvec(ctx, keys, v, layer["w_b"], plan_b, layer)

    # Algorithm 1
    xr = ckks.mul_plain(ctx, x, mask / (2.0 * R))
    for j in range(1, J + 1):
        xr = ckks.add(ctx, xr, ckks.rotate(ctx, keys, xr, -n_i * 2 ** (j - 1)))

    # Algorithm 2
    Gm = grid_matrix(layer)
    r = G + 2 * k + 1
    g1 = coltile(Gm, 1, r)
    g2 = coltile(Gm, 2, r + 1)
    if layer.get("b0") == "difference":
        # B_{m,0} = s_m - s_{m+1}, s_m = PolyComp(x - t_m) over the g + 2k + 1
        # knots: one comparison, and rot(s, n_i) brings block m + 1 to block
        # m (no product, one level fewer); block g + 2k is left with garbage
        # that the recursion's zero coefficients (or the k = 0 mask) remove
        g0 = coltile(Gm, 1, r + 1)
        s_ = polycomp0(ctx, keys, ckks.add_plain(ctx, xr, -g0 / (2.0 * R)), layer["comp"])
        b = ckks.sub(ctx, s_, ckks.rotate(ctx, keys, s_, n_i))
    else:
        a1 = ckks.add_plain(ctx, xr, -g1 / (2.0 * R))
        a2 = ckks.add_plain(ctx, ckks.mul_int(ctx, xr, -1), g2 / (2.0 * R))
        s1 = polycomp0(ctx, keys, a1, layer["comp"])
        s2 = polycomp0(ctx, keys, a2, layer["comp"])
        b = ckks.mul(ctx, keys, s1, s2)
    if k == 0:
        # order-0 basis: outside its n_i g valid slots b holds leftovers
        # (PolyComp(0)^2 = 1/4 in the product form), which the matvec's
        # replication would fold in; zero it (1 level)
        b = ckks.mul_plain(ctx, b, np.ones(n_i * G))
    for j in range(1, k + 1):
        t1 = coltile(Gm, 1, r - j)
        t2 = coltile(Gm, j + 1, r)
        t3 = coltile(Gm, j + 2, r + 1)
        t4 = coltile(Gm, 2, r - j + 1)
        A1 = 1.0 / (t2 - t1)
        A2 = 1.0 / (t3 - t4)
        lb = b.level
        xd = ckks.mod_drop(ctx, xr, lb + 1)
        u1 = ckks.add_plain(ctx, ckks.mul_plain(ctx, xd, 2.0 * R * A1), -t1 * A1)
        u2 = ckks.add_plain(ctx, ckks.mul_plain(ctx, xd, -2.0 * R * A2), t3 * A2)
        rb = ckks.rotate(ctx, keys, b, n_i)
        b = ckks.mul_sum(ctx, keys, [(u1, b), (u2, rb)])

    plan_s = bsgs_plan(n_o, n_i * (G + k), S)
    if layer.get("naive"):
        # the naive method the paper compares against (Table 3): reorder the
        # ColTile basis to row-major by an HE matvec with the permutation P of
        # Algorithm 3, then multiply by W' (one more level, n_i(g+k) diagonals)
        n = n_i * (G + k)
        plan_p = bsgs_plan(n, n, S)
        if plan_p["npad"] < S:
            b = ckks.add(ctx, b, ckks.rotate(ctx, keys, b, -plan_p["npad"]))
        b = matvec(ctx, keys, b, permutation_matrix(n_i, G + k), plan_p, layer)
        Ws = lazy_weights(layer)
    else:
        # fused linear layer (Eq. 13)
        Ws = fused_weights(layer)
    if plan_s["npad"] < S:
        b = ckks.add(ctx, b, ckks.rotate(ctx, keys, b, -plan_s["npad"]))
    ys = matvec(ctx, keys, b, Ws, plan_s, layer)

    lv = min(ys.level, yb.level)
    return ckks.add(ctx, ckks.level_down(ctx, ys, lv), ckks.level_down(ctx, yb, lv))


def chunking(layer, slots):
    """(K, n_c): a layer whose repeat-packed input n_i 2^ceil(log2(g+2k))
    exceeds the slots takes K input ciphertexts of n_c = slots / 2^J inputs
    each (the last one zero-padded); otherwise (1, n_i)."""
    J = rep_bits(layer)
    cap = slots >> J
    n_i = layer["n_in"]
    if n_i <= cap:
        return 1, n_i
    return -(-n_i // cap), cap


def chunk_layer(layer, c, n_c):
    """The layer restricted to inputs [c n_c, (c+1) n_c), zero-padded."""
    n_i, n_o, nb = layer["n_in"], layer["n_out"], layer["G"] + layer["k"]
    sub = dict(layer)
    sub["n_in"] = n_c
    coef = np.zeros((n_o, n_c, nb))
    ws = np.zeros((n_o, n_c))
    wb = np.zeros((n_o, n_c))
    hi = min(n_i, (c + 1) * n_c)
    coef[:, : hi - c * n_c] = layer["coef"][:, c * n_c: hi]
    ws[:, : hi - c * n_c] = layer["w_s"][:, c * n_c: hi]
    wb[:, : hi - c * n_c] = layer["w_b"][:, c * n_c: hi]
    sub["coef"], sub["w_s"], sub["w_b"] = coef, ws, wb
    return sub


def layer_eval_chunked(ctx, keys, xs, layer):
    """Wide layer: chunk c (ciphertext xs[c]) goes through the layer with the
    column blocks of chunk c; the partial outputs are summed in chunk order."""
    K, n_c = chunking(layer, ctx.slots)
    if len(xs) != K:
        raise ValueError("layer needs %d input ciphertexts" % K)
    out = None
    for c in range(K):
        y = layer_eval(ctx, keys, xs[c], chunk_layer(layer, c, n_c))
        out = y if out is None else ckks.add(ctx, out, y)
    return out


def infer(ctx, keys, x, model):
    """x: one ciphertext, or the list of K chunk ciphertexts of a wide first layer."""
    h = x
    for layer in model:
        if isinstance(h, (list, tuple)):
            h = layer_eval_chunked(ctx, keys, list(h), layer)
        else:
            h = layer_eval(ctx, keys, h, layer)
    return h


def model_rotations(model, slots):
    s = set()
    for layer in model:
        s.update(layer_rotations(layer, slots))
    return sorted(s)
