// Encrypted KAN layer schedule (paper, Method section).
//
//  SiLU branch (Eqs. 11-12): y = x (x) (mask * 2/(hi-lo)) + mask * (-(hi+lo)/(hi-lo)),
//    replicated to the matvec period, the Chebyshev polynomial by baby/giant
//    steps, then W_b by BSGS.
//  Spline branch: Algorithm 1 (mask with 1/(2R) folded in, then doubling
//    rotations by -n_i 2^(j-1)), Algorithm 2 (PolyComp through a composite of
//    odd polynomials, minimax stages or f_n, whose last stage returns
//    (1+f)/2; B0 = x1 (x) x2, or the difference of neighbouring knot
//    comparisons s - rot(s, n_i); k recursion steps sharing one
//    relinearisation each), then W_f = W'P (Algorithm 3, Eq. 13) by BSGS.
//  Output: both branches moved to the lower level and added.
// Plaintext vectors are encoded once per (tag, level, scale) and cached on
// the device; a batch shares them.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <set>
#include <tuple>

#include "ops.h"

using namespace ck;

namespace {

int pow2ceil(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

struct Plan {
  int no = 1, npad = 1, g1 = 1, g2 = 1;
  std::vector<int> folds;
};

Plan bsgs_plan(int n_out, int n, int slots) {
  Plan p;
  p.no = pow2ceil(n_out);
  p.npad = pow2ceil(std::max(n, p.no));
  if (p.npad > slots) throw Error(CKKS_ERR_UNSUPPORTED, "matrix does not fit the slots");
  int lg = 0;
  while ((1 << lg) < p.no) lg++;
  p.g1 = 1 << ((lg + 1) / 2);
  p.g2 = p.no / p.g1;
  for (int s = p.npad / 2; s >= p.no; s /= 2) p.folds.push_back(s);
  return p;
}

// odd monomial coefficients of f_n(x) = sum_i 4^-i C(2i,i) x (1-x^2)^i
std::vector<double> fn_coeffs(int n) {
  auto C = [](int a, int b) {
    int64_t r = 1;
    for (int i = 1; i <= b; i++) r = r * (a - b + i) / i;
    return r;
  };
  std::vector<double> c(n + 1);
  for (int l = 0; l <= n; l++) {
    int64_t num = 0;
    for (int i = l; i <= n; i++) num += C(2 * i, i) * C(i, l) * ((int64_t)1 << (2 * (n - i)));
    if (l & 1) num = -num;
    c[l] = (double)num / (double)((int64_t)1 << (2 * n));
  }
  return c;
}

struct Layer {
  int n_in, n_out, G, k;
  double lo, hi, R, silu_lo, silu_hi;
  std::vector<double> coef, w_s, w_b, cheb, knots;
  std::vector<std::vector<double>> comp;  // composite stages, odd monomial coefficients
  int b0 = 0;  // order-0 basis: 0 product (Algorithm 2), 1 difference of knot comparisons
  int bsgs = 0;  // 0 hoisted baby steps, 1 double hoisting (baby steps kept in QP_l)
  // A wide first layer (n_in 2^ceil(log2(G+2k)) > N/2) takes K input
  // ciphertexts per request of n_c inputs each (the last zero-padded);
  // otherwise K = 1 and n_c = n_in. The schedule runs on n_c inputs.
  int K = 1, n_c = 0;
  // naive: the spline branch reorders the ColTile basis by an HE matvec
  // with the permutation P (plan_p) and diag_s then holds W' instead of W_f
  bool naive = false;
  Plan plan_b, plan_s, plan_p;
  std::vector<std::vector<double>> diag_b, diag_s;  // per chunk: [no][slots]
};

}  // namespace

namespace {
// One layer schedule captured into a CUDA graph for one input shape. The
// graph reads its input from `in` and writes its result to `out`; every
// temporary is allocated and freed inside the graph.
struct GraphEntry {
  int uses = 0;
  uint64_t eager_launches = 0;
  cudaGraphExec_t exec = nullptr;
  Ct in, out;
  uint64_t launches[K_KIND_COUNT] = {};
  std::vector<ProfRec> prof;  // event pairs recorded by the graph (profiled capture)
  GraphEntry() = default;
  GraphEntry(const GraphEntry&) = delete;
  GraphEntry& operator=(const GraphEntry&) = delete;
  ~GraphEntry() {
    if (exec) cudaGraphExecDestroy(exec);
    for (auto& r : prof) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
  }
};
// (layer, batch, level, scale bits, key set, profiled)
using GraphKey = std::tuple<int, size_t, int, uint64_t, const ckks_keys*, bool>;
}  // namespace

struct kan_model {
  Ctx* ctx;
  std::vector<Layer> layers;
  std::map<std::tuple<int, int, int, int, uint64_t>, std::unique_ptr<DevBuf>> pts;
  bool graphs = false;
  const ckks_boot* boot = nullptr;  // refresh between layers when levels run short (borrowed)
  std::map<GraphKey, std::unique_ptr<GraphEntry>> graph_cache;  // destroyed before pts
};

namespace {

uint64_t dbits(double d) {
  uint64_t u;
  memcpy(&u, &d, 8);
  return u;
}

// cached plaintext of make() at (layer, tag, sub, level, scale)
template <class F>
const uint64_t* cached_pt(kan_model& M, int layer, int tag, int sub, int level, double scale,
                          F&& make) {
  auto key = std::make_tuple(layer * 1000 + tag, sub, level, 0, dbits(scale));
  auto it = M.pts.find(key);
  if (it != M.pts.end()) return it->second->u64();
  std::vector<double> v = make();
  auto b = std::make_unique<DevBuf>(encode_vec(*M.ctx, v.data(), v.size(), level, scale));
  const uint64_t* p = b->u64();
  M.pts[key] = std::move(b);
  return p;
}

// the same over QP_level (double hoisting)
template <class F>
const uint64_t* cached_pt_qp(kan_model& M, int layer, int tag, int sub, int level, double scale,
                             F&& make) {
  auto key = std::make_tuple(layer * 1000 + tag, sub, level, 1, dbits(scale));
  auto it = M.pts.find(key);
  if (it != M.pts.end()) return it->second->u64();
  std::vector<double> v = make();
  auto b = std::make_unique<DevBuf>(encode_vec_qp(*M.ctx, v.data(), v.size(), level, scale));
  const uint64_t* p = b->u64();
  M.pts[key] = std::move(b);
  return p;
}

std::vector<double> coltile(const Layer& L, int l, int r) {
  // G matrix rows are identical knot vectors (uniform grid); columns l..r-1,
  // 1-indexed, each tiled over the n_c inputs one ciphertext carries
  std::vector<double> out;
  for (int c = l; c < r; c++)
    for (int i = 0; i < L.n_c; i++) out.push_back(L.knots[c - 1]);
  return out;
}

std::vector<double> diagonals(const std::vector<double>& M, int n_out, int n, const Plan& p,
                              int slots) {
  std::vector<double> Mp((size_t)p.no * p.npad, 0.0);
  for (int o = 0; o < n_out; o++)
    for (int i = 0; i < n; i++) Mp[(size_t)o * p.npad + i] = M[(size_t)o * n + i];
  std::vector<double> D((size_t)p.no * slots, 0.0);
  for (int t = 0; t < p.no; t++)
    for (int s = 0; s < p.npad; s++)
      D[(size_t)t * slots + s] = Mp[(size_t)(s % p.no) * p.npad + (s + t) % p.npad];
  return D;
}

enum Tag { T_SILU_MUL = 1, T_SILU_ADD, T_MASK_R, T_G1, T_G2, T_U1M, T_U1A, T_U2M, T_U2A, T_DIAG_B, T_DIAG_S,
           T_MASK_B0, T_DIAG_P, T_DIAG_W, T_G0 };

// ColTile blocks Algorithm 1 must provide: one per order-0 basis function
// (g + 2k), or one per knot (g + 2k + 1) for the difference form
int rep_blocks(const Layer& L) { return L.G + 2 * L.k + (L.b0 == 1 ? 1 : 0); }
int rep_bits(const Layer& L) {
  int J = 0;
  while ((1 << J) < rep_blocks(L)) J++;
  return J;
}

// accessor of diagonals precomputed per chunk as [no][slots]
auto stored_diag(const std::vector<std::vector<double>>& DC, int S) {
  return [&DC, S](int ch, int t, int s) { return DC[ch][(size_t)t * S + s]; };
}

// y = M v by baby-step giant-step over the extended diagonals dval(ch, t, s)
// (chunk ch, diagonal t, slot s); batch element b uses chunk b % nch
template <class DV>
Ct bsgs_matvec(kan_model& M, int li, int tag, const Plan& p, int nch, DV&& dval,
               const ckks_keys& keys, const ckks_ct& v) {
  Ctx& c = *M.ctx;
  const int S = (int)(c.N / 2);
  std::vector<int64_t> bs;
  for (int j = 0; j < p.g1; j++) bs.push_back(j);
  std::vector<Ct> baby = op_rotate_many(c, keys, v, bs);
  const int lv = v.level;
  const size_t rows = v.B * 2 * (lv + 1);
  Ct z;
  for (int i = 0; i < p.g2; i++) {
    const double Spt = plain_scale(c, v.scale, lv);
    Ct acc = ct_alloc(c, v.B, lv, v.scale * Spt);
    for (int j = 0; j < p.g1; j++) {
      const int t = p.g1 * i + j;
      std::vector<const uint64_t*> pts;
      for (int ch = 0; ch < nch; ch++) {
        pts.push_back(cached_pt(M, li, tag, t * 64 + ch, lv, Spt, [&] {
          std::vector<double> d(S);
          const int sh = p.g1 * i;
          for (int s = 0; s < S; s++) d[s] = dval(ch, t, ((s - sh) % S + S) % S);
          return d;
        }));
      }
      // batch element b uses the diagonals of its chunk b % K (grouped forms)
      if (j == 0) {
        if (nch == 1)
          k_mul_pt(c, baby[j]->d.u64(), pts[0], acc->d.u64(), rows, lv + 1);
        else
          k_mul_pt_grouped(c, baby[j]->d.u64(), pts, acc->d.u64(), v.B, lv + 1);
      } else if (nch == 1) {
        k_mul_pt_acc(c, baby[j]->d.u64(), pts[0], acc->d.u64(), rows, lv + 1);
      } else {
        k_mul_pt_acc_grouped(c, baby[j]->d.u64(), pts, acc->d.u64(), v.B, lv + 1);
      }
    }
    Ct inner = op_rescale(c, *acc);
    if (i > 0) inner = op_rotate(c, keys, *inner, (int64_t)p.g1 * i);
    z = z ? op_add(c, *z, *inner, false) : std::move(inner);
  }
  for (int s : p.folds) {
    Ct r = op_rotate(c, keys, *z, s);
    z = op_add(c, *z, *r, false);
  }
  return z;
}

// bsgs_matvec with double hoisting: the baby-step rotations stay in QP_l (one
// ModUp, no ModDown: R_j = (P sigma_j(c0) + acc_0, acc_1), R_0 = P v), each
// giant step's diagonal products are summed over QP_l with the diagonals
// encoded over QP_l, and the sum is divided by P q_level once (the ModDowns
// of the baby steps and the rescale of the products in one rounded
// division), then rotated by g1 i. One input chunk (nch = 1).
template <class DV>
Ct bsgs_matvec_double(kan_model& M, int li, int tag, const Plan& p, DV&& dval,
                      const ckks_keys& keys, const ckks_ct& v) {
  Ctx& c = *M.ctx;
  const int S = (int)(c.N / 2);
  const int lv = v.level, l = lv + 1;
  if (lv < 1) throw Error(CKKS_ERR_LEVEL, "level exhausted");
  ConvTables& T = c.tables(lv);
  const size_t qp_words = v.B * 2 * (size_t)T.rows * c.N;
  std::vector<DevBuf> R;
  R.emplace_back(&c, qp_words * 8);
  k_qp_lift(c, v.d.u64(), v.B, lv, nullptr, R[0].u64());
  DevBuf ext;
  for (int j = 1; j < p.g1; j++) {
    const uint64_t g = c.galois(j);
    DevBuf kt;
    const uint64_t* key = switch_key_words(c, keys, g, kt);
    if (!ext.p) {
      ext = DevBuf(&c, v.B * T.beta * T.rows * c.N * 8);
      // c1 of batch element b sits at v + (2b + 1) l N
      modup(c, v.d.u64() + (size_t)l * c.N, v.B, lv, ext.u64(), 2 * (size_t)l * c.N);
    }
    DevBuf acc = keyswitch_qp(c, ext.u64(), v.B, lv, key, g);
    k_qp_lift(c, v.d.u64(), v.B, lv, c.perm(g), acc.u64());
    R.push_back(std::move(acc));
  }
  ext.reset();
  const double Spt = plain_scale(c, v.scale, lv);
  double s = v.scale * Spt / (double)c.mod[lv];
  if (fabs(s / c.delta[lv - 1] - 1.0) < SNAP) s = c.delta[lv - 1];
  Ct z;
  for (int i = 0; i < p.g2; i++) {
    DevBuf acc(&c, qp_words * 8);
    for (int j = 0; j < p.g1; j++) {
      const int t = p.g1 * i + j;
      const uint64_t* pt = cached_pt_qp(M, li, tag, t * 64, lv, Spt, [&] {
        std::vector<double> d(S);
        const int sh = p.g1 * i;
        for (int q = 0; q < S; q++) d[q] = dval(0, t, ((q - sh) % S + S) % S);
        return d;
      });
      k_qp_mul_pt_acc(c, R[j].u64(), pt, acc.u64(), v.B * 2, lv, j == 0);
    }
    Ct inner = ct_alloc(c, v.B, lv - 1, s);
    div_p_ql(c, acc.u64(), v.B, lv, inner->d.u64());
    if (i > 0) inner = op_rotate(c, keys, *inner, (int64_t)p.g1 * i);
    z = z ? op_add(c, *z, *inner, false) : std::move(inner);
  }
  for (int f : p.folds) {
    Ct r = op_rotate(c, keys, *z, f);
    z = op_add(c, *z, *r, false);
  }
  return z;
}

// the layer's matvec form; double hoisting takes one input chunk
template <class DV>
Ct matvec(kan_model& M, int li, int tag, const Plan& p, int nch, DV&& dval, const ckks_keys& keys,
          const ckks_ct& v) {
  if (M.layers[li].bsgs == 1) {
    if (nch != 1) throw Error(CKKS_ERR_UNSUPPORTED, "double hoisting of a chunked layer");
    return bsgs_matvec_double(M, li, tag, p, dval, keys, v);
  }
  return bsgs_matvec(M, li, tag, p, nch, dval, keys, v);
}

// sum_l cf[l] u^(2l+1) + cst: the coefficients, padded to 2^K, split in
// halves, p = A + u^(2^K) B with A and B the odd polynomials of the lower and
// upper halves, recursively; one coefficient is a constant product. Depth
// K + 1 = ceil(log2(degree + 1)); f_3 takes 5 ciphertext products.
Ct odd_split(Ctx& c, const ckks_keys& keys, const ckks_ct& u, const std::vector<double>& cf,
             const std::vector<Ct>& pw, int lo, int k) {
  if (k == 0) return cf[lo] != 0.0 ? op_mul_const(c, u, cf[lo]) : Ct();
  const int half = 1 << (k - 1);
  Ct A = odd_split(c, keys, u, cf, pw, lo, k - 1);
  Ct B = odd_split(c, keys, u, cf, pw, lo + half, k - 1);
  if (!B) return A;
  Ct P = op_mul(c, keys, *B, *pw[k]);
  if (!A) return P;
  Ct Ad = op_level_down(c, *A, P->level);
  return op_add(c, *Ad, *P, false);
}

Ct eval_odd(Ctx& c, const ckks_keys& keys, const ckks_ct& u, const std::vector<double>& cf0,
            double cst) {
  int K = 0;
  while ((size_t)1 << K < cf0.size()) K++;
  std::vector<double> cf(cf0);
  cf.resize((size_t)1 << K, 0.0);
  std::vector<Ct> pw(K + 1);  // pw[k] = u^(2^k), k >= 1
  for (int k = 1; k <= K; k++) {
    const ckks_ct& h = k == 1 ? u : *pw[k - 1];
    pw[k] = op_mul(c, keys, h, h);
  }
  Ct out = odd_split(c, keys, u, cf, pw, 0, K);
  if (!out) throw Error(CKKS_ERR_INVALID_ARG, "comparison polynomial without coefficients");
  if (cst != 0.0) out = op_add_const(c, *out, cst);
  return out;
}

Ct polycomp0(Ctx& c, const ckks_keys& keys, const ckks_ct& a,
              const std::vector<std::vector<double>>& stages) {
  Ct u;
  const ckks_ct* cur = &a;
  for (size_t s = 0; s < stages.size(); s++) {
    std::vector<double> cf = stages[s];
    if (s + 1 == stages.size()) {
      for (auto& x : cf) x = 0.5 * x;
      u = eval_odd(c, keys, *cur, cf, 0.5);
    } else {
      u = eval_odd(c, keys, *cur, cf, 0.0);
    }
    cur = u.get();
  }
  return u;
}

Ct eval_cheb(Ctx& c, const ckks_keys& keys, const ckks_ct& y, const std::vector<double>& a) {
  const int d = (int)a.size() - 1;
  const int m = pow2ceil((int)ceil(sqrt((double)(d + 1))));
  std::map<int, Ct> T;
  T[1] = ct_copy(c, y);
  for (int i = 2; i <= m; i++) {
    if ((i & (i - 1)) == 0) {
      Ct sq = op_mul(c, keys, *T[i / 2], *T[i / 2]);
      T[i] = op_add_const(c, *op_mul_int(c, *sq, 2), -1.0);
    } else {
      int hb = 1;
      while (hb * 2 <= i) hb *= 2;
      const int lo = i - hb;
      Ct pr = op_mul_int(c, *op_mul(c, keys, *T[hb], *T[lo]), 2);
      if (hb - lo == 0)
        T[i] = op_add_const(c, *pr, -1.0);
      else
        T[i] = op_add(c, *pr, *op_level_down(c, *T[hb - lo], pr->level), true);
    }
  }
  std::map<int, Ct> Gs;
  Gs[m] = ct_copy(c, *T[m]);
  int D = m;
  while (2 * D <= d) {
    Ct sq = op_mul(c, keys, *Gs[D], *Gs[D]);
    Gs[2 * D] = op_add_const(c, *op_mul_int(c, *sq, 2), -1.0);
    D *= 2;
  }
  struct R {
    Ct ct;
    double v;
  };
  std::function<R(const std::vector<double>&)> rec = [&](const std::vector<double>& cf) -> R {
    const int deg = (int)cf.size() - 1;
    if (deg < m) {
      if (deg == 0) return R{nullptr, cf[0]};
      std::vector<const ckks_ct*> in;
      std::vector<double> k;
      for (int i = 1; i <= deg; i++) {
        in.push_back(T[i].get());
        k.push_back(cf[i]);
      }
      return R{op_lincomb(c, in, k, cf[0], -1), 0.0};
    }
    int Dd = m;
    while (2 * Dd <= deg) Dd *= 2;
    std::vector<double> q;
    q.push_back(cf[Dd]);
    for (int i = 1; i <= deg - Dd; i++) q.push_back(2.0 * cf[Dd + i]);
    std::vector<double> r(cf.begin(), cf.begin() + Dd);
    for (int i = 1; i <= deg - Dd; i++) r[Dd - i] -= cf[Dd + i];
    R Q = rec(q);
    R Rr = rec(r);
    Ct P;
    if (!Q.ct)
      P = op_lincomb(c, {Gs[Dd].get()}, {Q.v}, 0.0, -1);
    else
      P = op_mul(c, keys, *Q.ct, *Gs[Dd]);
    if (!Rr.ct) return R{op_add_const(c, *P, Rr.v), 0.0};
    const int lv = std::min(P->level, Rr.ct->level);
    return R{op_add(c, *op_level_down(c, *P, lv), *op_level_down(c, *Rr.ct, lv), false), 0.0};
  };
  R out = rec(a);
  if (!out.ct) throw Error(CKKS_ERR_INVALID_ARG, "SiLU polynomial of degree 0");
  return std::move(out.ct);
}

Ct layer_eval(kan_model& M, int li, const ckks_keys& keys, const ckks_ct& x) {
  Ctx& c = *M.ctx;
  Layer& L = M.layers[li];
  const int S = (int)(c.N / 2);
  const int n_i = L.n_c, G = L.G, k = L.k;  // inputs per ciphertext
  const double R = L.R;
  const int J = rep_bits(L);
  if ((int64_t)n_i << J > S) throw Error(CKKS_ERR_UNSUPPORTED, "n_i * 2^J > N/2 (Algorithm 1)");
  if (x.level < 1) throw Error(CKKS_ERR_LEVEL, "level exhausted");
  if (x.B % L.K != 0) throw Error(CKKS_ERR_INVALID_ARG, "batch is not a multiple of the layer's chunks");

  // SiLU branch
  const double sa = 2.0 / (L.silu_hi - L.silu_lo), sb = -(L.silu_hi + L.silu_lo) / (L.silu_hi - L.silu_lo);
  const double S1 = plain_scale(c, x.scale, x.level);
  const uint64_t* p_sm = cached_pt(M, li, T_SILU_MUL, 0, x.level, S1,
                                   [&] { return std::vector<double>(n_i, sa * 1.0); });
  Ct y0 = op_mul_pt(c, x, p_sm, S1);
  const uint64_t* p_sa = cached_pt(M, li, T_SILU_ADD, 0, y0->level, y0->scale,
                                   [&] { return std::vector<double>(n_i, sb * 1.0); });
  Ct y = op_add_pt(c, *y0, p_sa);
  if (L.plan_b.npad < S) y = op_add(c, *y, *op_rotate(c, keys, *y, -L.plan_b.npad), false);
  Ct v = eval_cheb(c, keys, *y, L.cheb);
  Ct yb = matvec(M, li, T_DIAG_B, L.plan_b, L.K, stored_diag(L.diag_b, S), keys, *v);

  // Algorithm 1
  const uint64_t* p_mr = cached_pt(M, li, T_MASK_R, 0, x.level, S1,
                                   [&] { return std::vector<double>(n_i, 1.0 / (2.0 * R)); });
  Ct xr = op_mul_pt(c, x, p_mr, S1);
  for (int j = 1; j <= J; j++)
    xr = op_add(c, *xr, *op_rotate(c, keys, *xr, -(int64_t)n_i * (1 << (j - 1))), false);

  // Algorithm 2
  const int r = G + 2 * k + 1;
  Ct b;
  if (L.b0 == 1) {
    // B_{m,0} = s_m - s_{m+1}, s_m = PolyComp(x - t_m) against every knot
    // (block m compares with t_m): one comparison, and rot(s, n_i) brings
    // block m + 1 to block m (no product, one level fewer); the last block
    // is left with leftovers that the recursion's zero coefficients (or the
    // k = 0 mask) remove
    const uint64_t* p_g0 = cached_pt(M, li, T_G0, 0, xr->level, xr->scale, [&] {
      std::vector<double> g0 = coltile(L, 1, r + 1);
      for (auto& t : g0) t = -t / (2.0 * R);
      return g0;
    });
    Ct a0 = op_add_pt(c, *xr, p_g0);
    Ct s0 = polycomp0(c, keys, *a0, L.comp);
    b = op_add(c, *s0, *op_rotate(c, keys, *s0, n_i), true);
  } else {
    const uint64_t* p_g1 = cached_pt(M, li, T_G1, 0, xr->level, xr->scale, [&] {
      std::vector<double> g1 = coltile(L, 1, r);
      for (auto& t : g1) t = -t / (2.0 * R);
      return g1;
    });
    Ct a1 = op_add_pt(c, *xr, p_g1);
    const uint64_t* p_g2 = cached_pt(M, li, T_G2, 0, xr->level, xr->scale, [&] {
      std::vector<double> g2 = coltile(L, 2, r + 1);
      for (auto& t : g2) t = t / (2.0 * R);
      return g2;
    });
    Ct a2 = op_add_pt(c, *op_mul_int(c, *xr, -1), p_g2);
    Ct s1 = polycomp0(c, keys, *a1, L.comp);
    Ct s2 = polycomp0(c, keys, *a2, L.comp);
    b = op_mul(c, keys, *s1, *s2);
  }
  if (k == 0) {
    // order-0 basis: outside its n_i g valid slots b holds leftovers
    // (PolyComp(0)^2 = 1/4 in the product form), which the matvec's
    // replication would fold in; zero it (1 level)
    const double Sb = plain_scale(c, b->scale, b->level);
    const uint64_t* p_b0 = cached_pt(M, li, T_MASK_B0, 0, b->level, Sb,
                                     [&] { return std::vector<double>((size_t)n_i * G, 1.0); });
    b = op_mul_pt(c, *b, p_b0, Sb);
  }
  for (int j = 1; j <= k; j++) {
    const std::vector<double> t1 = coltile(L, 1, r - j), t2 = coltile(L, j + 1, r);
    const std::vector<double> t3 = coltile(L, j + 2, r + 1), t4 = coltile(L, 2, r - j + 1);
    std::vector<double> A1(t1.size()), A2(t3.size());
    for (size_t i = 0; i < t1.size(); i++) A1[i] = 1.0 / (t2[i] - t1[i]);
    for (size_t i = 0; i < t3.size(); i++) A2[i] = 1.0 / (t3[i] - t4[i]);
    const int lb = b->level;
    Ct xd = op_mod_drop(c, *xr, lb + 1);
    const double Su = plain_scale(c, xd->scale, xd->level);
    const uint64_t* p1m = cached_pt(M, li, T_U1M, j, xd->level, Su, [&] {
      std::vector<double> v2(A1.size());
      for (size_t i = 0; i < A1.size(); i++) v2[i] = 2.0 * R * A1[i];
      return v2;
    });
    Ct u1 = op_mul_pt(c, *xd, p1m, Su);
    const uint64_t* p1a = cached_pt(M, li, T_U1A, j, u1->level, u1->scale, [&] {
      std::vector<double> v2(A1.size());
      for (size_t i = 0; i < A1.size(); i++) v2[i] = -t1[i] * A1[i];
      return v2;
    });
    u1 = op_add_pt(c, *u1, p1a);
    const uint64_t* p2m = cached_pt(M, li, T_U2M, j, xd->level, Su, [&] {
      std::vector<double> v2(A2.size());
      for (size_t i = 0; i < A2.size(); i++) v2[i] = -2.0 * R * A2[i];
      return v2;
    });
    Ct u2 = op_mul_pt(c, *xd, p2m, Su);
    const uint64_t* p2a = cached_pt(M, li, T_U2A, j, u2->level, u2->scale, [&] {
      std::vector<double> v2(A2.size());
      for (size_t i = 0; i < A2.size(); i++) v2[i] = t3[i] * A2[i];
      return v2;
    });
    u2 = op_add_pt(c, *u2, p2a);
    Ct rb = op_rotate(c, keys, *b, n_i);
    b = op_mul_sum(c, keys, {{u1.get(), b.get()}, {u2.get(), rb.get()}});
  }

  if (L.naive) {
    // the naive method: reorder the ColTile basis to row-major by an HE
    // matvec with the permutation P of Algorithm 3, shared by every chunk
    if (L.plan_p.npad < S) b = op_add(c, *b, *op_rotate(c, keys, *b, -L.plan_p.npad), false);
    const int nb = G + k, n = n_i * nb, npad = L.plan_p.npad, no = L.plan_p.no;
    auto perm = [=](int, int t, int s) -> double {
      if (s >= npad) return 0.0;
      const int r = s % no, col = (s + t) % npad;  // P[r][col]
      if (r >= n || col >= n) return 0.0;
      return col == (r % nb) * n_i + r / nb ? 1.0 : 0.0;
    };
    b = matvec(M, li, T_DIAG_P, L.plan_p, 1, perm, keys, *b);
  }
  // fused linear layer W_f (Eq. 13), or W' after the naive permutation
  if (L.plan_s.npad < S) b = op_add(c, *b, *op_rotate(c, keys, *b, -L.plan_s.npad), false);
  Ct ys = matvec(M, li, L.naive ? T_DIAG_W : T_DIAG_S, L.plan_s, L.K, stored_diag(L.diag_s, S),
                 keys, *b);
  const int lv = std::min(ys->level, yb->level);
  Ct out = op_add(c, *op_level_down(c, *ys, lv), *op_level_down(c, *yb, lv), false);
  if (L.K == 1) return out;
  // chunk partial outputs b*K + ch summed in chunk order
  Ct sum = ct_alloc(c, out->B / L.K, out->level, out->scale);
  k_chunk_sum(c, out->d.u64(), sum->d.u64(), sum->B, L.K, out->level + 1);
  return sum;
}

// Capture layer li's schedule on input shape x into g (the plaintext cache
// and the conversion tables are already filled by an eager run).
void capture_layer(kan_model& M, int li, const ckks_keys& keys, const ckks_ct& x, GraphEntry& g) {
  Ctx& c = *M.ctx;
  g.in = ct_alloc(c, x.B, x.level, x.scale);
  if (c.prof) {  // events for the record nodes, created before the capture
    std::vector<cudaEvent_t> ev;
    for (uint64_t i = 0; i < 2 * g.eager_launches; i++) ev.push_back(c.take_event());
    for (cudaEvent_t e : ev) c.ev_pool.push_back(e);
  }
  uint64_t before[K_KIND_COUNT];
  memcpy(before, c.launches, sizeof(before));
  std::vector<ProfRec> recs;
  c.prof_sink = &recs;
  cudaGraph_t graph = nullptr;
  CK_CUDA(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
  try {
    Ct y = layer_eval(M, li, keys, *g.in);
    if (y->B != g.out->B || y->level != g.out->level || y->scale != g.out->scale)
      throw Error(CKKS_ERR_CUDA, "layer output shape differs between runs");
    CK_CUDA(cudaMemcpyAsync(g.out->d.p, y->d.p, y->d.bytes, cudaMemcpyDeviceToDevice, c.stream));
    y.reset();
    CK_CUDA(cudaStreamEndCapture(c.stream, &graph));
  } catch (...) {
    cudaGraph_t junk = nullptr;
    cudaStreamEndCapture(c.stream, &junk);
    if (junk) cudaGraphDestroy(junk);
    cudaGetLastError();
    c.prof_sink = nullptr;
    memcpy(c.launches, before, sizeof(before));
    for (auto& r : recs) {
      c.ev_pool.push_back(r.a);
      c.ev_pool.push_back(r.b);
    }
    throw;
  }
  c.prof_sink = nullptr;
  for (int k = 0; k < K_KIND_COUNT; k++) {
    g.launches[k] = c.launches[k] - before[k];
    c.launches[k] = before[k];
  }
  g.prof = std::move(recs);
  const cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  CK_CUDA(e);
}

// Layer li on x: eager, or with graphs on, replayed from the graph captured
// for x's shape (first call of a shape eager, second captures). Replays
// compute exactly what the eager schedule computes.
Ct layer_run(kan_model& M, int li, const ckks_keys& keys, const ckks_ct& x) {
  if (!M.graphs) return layer_eval(M, li, keys, x);
  Ctx& c = *M.ctx;
  auto& slot = M.graph_cache[GraphKey(li, x.B, x.level, dbits(x.scale), &keys, c.prof)];
  if (!slot) slot = std::make_unique<GraphEntry>();
  GraphEntry& g = *slot;
  if (g.uses++ == 0) {
    uint64_t n0 = 0, n1 = 0;
    for (int k = 0; k < K_KIND_COUNT; k++) n0 += c.launches[k];
    Ct y = layer_eval(M, li, keys, x);
    for (int k = 0; k < K_KIND_COUNT; k++) n1 += c.launches[k];
    g.eager_launches = n1 - n0;
    g.out = ct_alloc(c, y->B, y->level, y->scale);
    return y;
  }
  if (!g.exec) capture_layer(M, li, keys, x, g);
  {
    Launch L_(c, K_COPY, 2.0 * (double)x.d.bytes);
    CK_CUDA(cudaMemcpyAsync(g.in->d.p, x.d.p, x.d.bytes, cudaMemcpyDeviceToDevice, c.stream));
  }
  CK_CUDA(cudaGraphLaunch(g.exec, c.stream));
  for (int k = 0; k < K_KIND_COUNT; k++) c.launches[k] += g.launches[k];
  if (c.prof && !g.prof.empty()) {
    CK_CUDA(cudaStreamSynchronize(c.stream));
    for (const ProfRec& r : g.prof) {
      float t = 0;
      CK_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
      c.prof_acc[r.kind][0] += t;
      c.prof_acc[r.kind][1] += r.bytes;
      c.prof_acc[r.kind][2] += r.ops;
      c.prof_acc[r.kind][3] += 1;
    }
  }
  Ct r = ct_alloc(c, g.out->B, g.out->level, g.out->scale);
  Launch L_(c, K_COPY, 2.0 * (double)r->d.bytes);
  CK_CUDA(cudaMemcpyAsync(r->d.p, g.out->d.p, r->d.bytes, cudaMemcpyDeviceToDevice, c.stream));
  return r;
}

int cheb_depth(int d) {
  const int m = pow2ceil((int)ceil(sqrt((double)(d + 1))));
  std::map<int, int> T;
  T[1] = 0;
  for (int i = 2; i <= m; i++) {
    if ((i & (i - 1)) == 0) {
      T[i] = T[i / 2] + 1;
    } else {
      int hb = 1;
      while (hb * 2 <= i) hb *= 2;
      T[i] = std::max(T[hb], T[i - hb]) + 1;
    }
  }
  std::map<int, int> Gs;
  Gs[m] = T[m];
  for (int D = m; 2 * D <= d; D *= 2) Gs[2 * D] = Gs[D] + 1;
  std::function<int(int)> rec = [&](int deg) -> int {  // -1 = constant
    if (deg < m) {
      if (deg == 0) return -1;
      int mx = 0;
      for (int i = 1; i <= deg; i++) mx = std::max(mx, T[i]);
      return mx + 1;
    }
    int D = m;
    while (2 * D <= deg) D *= 2;
    const int q = rec(deg - D), r = rec(D - 1);
    const int P = q < 0 ? Gs[D] + 1 : std::max(q, Gs[D]) + 1;
    return r < 0 ? P : std::max(P, r);
  };
  return rec(d);
}

int layer_depth(const Layer& L) {
  int dc = 0;
  for (const auto& st : L.comp) {  // an odd polynomial of 2^K coefficients: depth K + 1
    int K = 0;
    while (((size_t)1 << K) < st.size()) K++;
    dc += K + 1;
  }
  // mask, comparison, B0 product (not in the difference form), recursion
  // (k = 0 masks its basis instead of a recursion step), naive P matvec, W_f
  const int spline = 1 + dc + (L.b0 == 1 ? 0 : 1) + std::max(L.k, 1) + (L.naive ? 1 : 0) + 1;
  const int silu = 2 + cheb_depth((int)L.cheb.size() - 1);
  return std::max(spline, silu);
}

std::vector<int> layer_rotations(const Layer& L, int slots) {
  std::set<int> s;
  const int J = rep_bits(L);
  for (int j = 1; j <= J; j++) s.insert(-L.n_c * (1 << (j - 1)));
  s.insert(L.n_c);
  const int n_s = L.n_c * (L.G + L.k);
  std::vector<std::pair<int, int>> shapes = {{L.n_out, n_s}, {L.n_out, L.n_c}};
  if (L.naive) shapes.push_back({n_s, n_s});
  for (auto sh : shapes) {
    Plan p = bsgs_plan(sh.first, sh.second, slots);
    if (p.npad < slots) s.insert(-p.npad);
    for (int j = 1; j < p.g1; j++) s.insert(j);
    for (int i = 1; i < p.g2; i++) s.insert(p.g1 * i);
    for (int f : p.folds) s.insert(f);
  }
  s.erase(0);
  return std::vector<int>(s.begin(), s.end());
}

}  // namespace

// internal entry points for the serving scheduler
namespace ck {
Ct kan_eval_layer(kan_model& M, int layer, const ckks_keys& keys, const ckks_ct& x) {
  return layer_run(M, layer, keys, x);
}
int kan_num_layers(const kan_model& M) { return (int)M.layers.size(); }
int kan_layer_chunks(const kan_model& M, int layer) { return M.layers[layer].K; }
int kan_total_depth(const kan_model& M) {
  int d = 0;
  for (const Layer& L : M.layers) d += layer_depth(L);
  return d;
}
// the level an input needs: the whole network's depth, or with a
// bootstrapping plan the first layer's (later layers run on refreshes)
int kan_input_depth(const kan_model& M) {
  return M.boot ? layer_depth(M.layers[0]) : kan_total_depth(M);
}
// A layer after the first that needs more levels than are left runs on the
// refreshed batch: packed into as few ciphertexts as the slots allow when
// there are several and a level is left for the mask, else each brought to
// level 0 and bootstrapped; without a plan, or with levels enough, x as is.
Ct kan_refresh_for_layer(kan_model& M, int layer, const ckks_keys& keys, Ct x) {
  if (layer == 0 || !M.boot || x->level >= layer_depth(M.layers[layer])) return x;
  Ctx& c = *M.ctx;
  if (x->B > 1 && x->level >= 1)
    return refresh_packed(c, keys, *M.boot, *x, M.layers[layer - 1].n_out);
  Ct low = op_level_down(c, *x, 0);
  return bootstrap(c, keys, *M.boot, *low);
}
Ct cheb_eval(Ctx& c, const ckks_keys& keys, const ckks_ct& y, const std::vector<double>& a) {
  return eval_cheb(c, keys, y, a);
}
int cheb_levels(int degree) { return cheb_depth(degree); }
}  // namespace ck

extern "C" {

int kan_model_create(ckks_ctx* ctx, const kan_layer_desc* layers, size_t n_layers,
                     kan_model** out) {
  try {
    if (!ctx || !layers || !out || n_layers == 0) throw Error(CKKS_ERR_INVALID_ARG, "bad argument");
    auto M = std::make_unique<kan_model>();
    M->ctx = &ctx->c;
    const int S = (int)(ctx->c.N / 2);
    for (size_t li = 0; li < n_layers; li++) {
      const kan_layer_desc& d = layers[li];
      if (d.n_in < 1 || d.n_out < 1 || d.G < 1 || d.k < 0 || !d.coef || !d.w_s || !d.w_b ||
          !d.silu_cheb || d.silu_degree < 1 || !(d.R > 0) || !(d.silu_hi > d.silu_lo) ||
          !(d.grid_hi > d.grid_lo) || (d.b0_form != 0 && d.b0_form != 1) ||
          (d.bsgs_form != 0 && d.bsgs_form != 1))
        throw Error(CKKS_ERR_INVALID_ARG, "invalid layer description");
      Layer L;
      if (d.n_comp_poly > 0) {
        if (!d.comp_poly || !d.comp_poly_len)
          throw Error(CKKS_ERR_INVALID_ARG, "comparison stages without coefficients");
        const double* cp = d.comp_poly;
        for (int s = 0; s < d.n_comp_poly; s++) {
          const int n = d.comp_poly_len[s];
          if (n < 1 || n > 32) throw Error(CKKS_ERR_INVALID_ARG, "a comparison stage needs 1..32 coefficients");
          L.comp.emplace_back(cp, cp + n);
          cp += n;
        }
      } else {
        if (!d.comp || d.n_comp < 1) throw Error(CKKS_ERR_INVALID_ARG, "no comparison composite");
        for (int i = 0; i < d.n_comp; i++) {
          if (d.comp[i] < 1 || d.comp[i] > 8)
            throw Error(CKKS_ERR_INVALID_ARG, "comparison orders must be 1..8");
          L.comp.push_back(fn_coeffs(d.comp[i]));
        }
      }
      L.b0 = d.b0_form;
      L.bsgs = d.bsgs_form;
      L.n_in = d.n_in;
      L.n_out = d.n_out;
      L.G = d.G;
      L.k = d.k;
      L.lo = d.grid_lo;
      L.hi = d.grid_hi;
      L.R = d.R;
      L.silu_lo = d.silu_lo;
      L.silu_hi = d.silu_hi;
      const size_t nb = (size_t)d.G + d.k;
      L.coef.assign(d.coef, d.coef + (size_t)d.n_out * d.n_in * nb);
      L.w_s.assign(d.w_s, d.w_s + (size_t)d.n_out * d.n_in);
      L.w_b.assign(d.w_b, d.w_b + (size_t)d.n_out * d.n_in);
      L.cheb.assign(d.silu_cheb, d.silu_cheb + d.silu_degree + 1);
      const double h = (L.hi - L.lo) / L.G;
      for (int m = 0; m <= L.G + 2 * L.k; m++) L.knots.push_back(L.lo + (double)(m - L.k) * h);
      const int cap = S >> rep_bits(L);
      if (L.n_in <= cap) {
        L.K = 1;
        L.n_c = L.n_in;
      } else {
        if (li != 0)  // only the client can split an input
          throw Error(CKKS_ERR_UNSUPPORTED, "a hidden layer does not fit the slots");
        L.K = (L.n_in + cap - 1) / cap;
        L.n_c = cap;
        if (L.K > 16) throw Error(CKKS_ERR_UNSUPPORTED, "more than 16 input chunks");
      }
      // per chunk ch (inputs ch*n_c + i, zero beyond n_in): W_b columns and
      // W_f[o][m n_c + i] = w_s[o][i] c[o][i][m]  (W' P, Algorithm 3 / Eq. 13)
      const int n_c = L.n_c;
      const int n_s = n_c * (int)nb;
      L.naive = d.naive != 0;
      L.plan_b = bsgs_plan(d.n_out, n_c, S);
      L.plan_s = bsgs_plan(d.n_out, n_s, S);
      if (L.naive) L.plan_p = bsgs_plan(n_s, n_s, S);
      for (int ch = 0; ch < L.K; ch++) {
        std::vector<double> Wb((size_t)d.n_out * n_c, 0.0), Wf((size_t)d.n_out * n_s, 0.0);
        for (int o = 0; o < d.n_out; o++)
          for (int i = 0; i < n_c; i++) {
            const int gi = ch * n_c + i;
            if (gi >= d.n_in) continue;
            Wb[(size_t)o * n_c + i] = L.w_b[(size_t)o * d.n_in + gi];
            for (size_t m = 0; m < nb; m++)  // W' is row-major in (i, m), W_f ColTile
              Wf[(size_t)o * n_s + (L.naive ? i * nb + m : m * n_c + i)] =
                  L.w_s[(size_t)o * d.n_in + gi] * L.coef[((size_t)o * d.n_in + gi) * nb + m];
          }
        L.diag_b.push_back(diagonals(Wb, d.n_out, n_c, L.plan_b, S));
        L.diag_s.push_back(diagonals(Wf, d.n_out, n_s, L.plan_s, S));
      }
      M->layers.push_back(std::move(L));
    }
    *out = M.release();
    return CKKS_OK;
  } catch (...) {
    return api_error();
  }
}

int kan_model_destroy(kan_model* model) {
  delete model;
  return CKKS_OK;
}

int kan_model_rotations(const kan_model* model, int32_t* steps, size_t cap, size_t* n) {
  if (!model || !n) return CKKS_ERR_INVALID_ARG;
  std::set<int> s;
  for (const Layer& L : model->layers)
    for (int t : layer_rotations(L, (int)(model->ctx->N / 2))) s.insert(t);
  *n = s.size();
  size_t i = 0;
  for (int t : s) {
    if (i >= cap) break;
    if (steps) steps[i] = t;
    i++;
  }
  return CKKS_OK;
}

int kan_model_layer_depth(const kan_model* model, int layer, int* depth) {
  if (!model || !depth || layer < 0 || layer >= (int)model->layers.size()) return CKKS_ERR_INVALID_ARG;
  *depth = layer_depth(model->layers[layer]);
  return CKKS_OK;
}

int kan_model_set_bootstrap(kan_model* model, const ckks_boot* boot) {
  if (!model) return CKKS_ERR_INVALID_ARG;
  model->boot = boot;
  return CKKS_OK;
}

int kan_model_refresh_rotations(const kan_model* model, size_t batch, int32_t* steps, size_t cap,
                                size_t* n) {
  if (!model || !n || (cap && !steps)) return CKKS_ERR_INVALID_ARG;
  const int64_t S = (int64_t)model->ctx->N / 2;
  std::set<int64_t> st;
  for (size_t li = 1; li < model->layers.size(); li++) {
    int64_t nb = 1;
    while (nb < model->layers[li - 1].n_out) nb *= 2;
    const int64_t per = std::min<int64_t>(S / nb, (int64_t)batch);
    for (int64_t s = 1; s < per; s *= 2) {
      st.insert((s * nb) % S);
      st.insert(((-s * nb) % S + S) % S);
    }
  }
  st.erase(0);
  *n = st.size();
  size_t i = 0;
  for (int64_t v : st)
    if (i < cap) steps[i++] = (int32_t)v;
  return CKKS_OK;
}

int kan_model_set_graphs(kan_model* model, int enabled) {
  try {
    if (!model) return CKKS_ERR_INVALID_ARG;
    CK_CUDA(cudaStreamSynchronize(model->ctx->stream));
    model->graphs = enabled != 0;
    if (!model->graphs) model->graph_cache.clear();
    return CKKS_OK;
  } catch (...) {
    return api_error();
  }
}

int kan_model_layer_chunks(const kan_model* model, int layer, int* K, int* n_c) {
  if (!model || !K || !n_c || layer < 0 || layer >= (int)model->layers.size())
    return CKKS_ERR_INVALID_ARG;
  *K = model->layers[layer].K;
  *n_c = model->layers[layer].n_c;
  return CKKS_OK;
}

int kan_layer_eval(ckks_ctx* ctx, const ckks_keys* keys, kan_model* model, int layer,
                   const ckks_ct* in, ckks_ct** out) {
  try {
    if (!ctx || !keys || !model || !in || !out || layer < 0 || layer >= (int)model->layers.size())
      return CKKS_ERR_INVALID_ARG;
    *out = layer_run(*model, layer, *keys, *in).release();
    return CKKS_OK;
  } catch (...) {
    return api_error();
  }
}

int kan_infer(ckks_ctx* ctx, const ckks_keys* keys, kan_model* model, const ckks_ct* const* in,
              size_t n_in, ckks_ct** out) {
  try {
    if (!ctx || !keys || !model || !in || !out || n_in == 0) return CKKS_ERR_INVALID_ARG;
    Ctx& c = ctx->c;
    int lv = in[0]->level;
    for (size_t i = 0; i < n_in; i++) lv = std::min(lv, in[i]->level);
    std::vector<Ct> aligned;
    std::vector<const ckks_ct*> parts;
    for (size_t i = 0; i < n_in; i++) {
      if (in[i]->level != lv) {
        aligned.push_back(op_level_down(c, *in[i], lv));
        parts.push_back(aligned.back().get());
      } else {
        parts.push_back(in[i]);
      }
    }
    Ct h = parts.size() == 1 ? ct_copy(c, *parts[0]) : op_concat(c, parts);
    aligned.clear();
    for (size_t li = 0; li < model->layers.size(); li++) {
      h = kan_refresh_for_layer(*model, (int)li, *keys, std::move(h));
      h = layer_run(*model, (int)li, *keys, *h);
    }
    *out = h.release();
    return CKKS_OK;
  } catch (...) {
    return api_error();
  }
}

}  // extern "C"
