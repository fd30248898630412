// CKKS bootstrapping: ModRaise, CoeffToSlot, EvalMod, SlotToCoeff.
//
// The paper's parameter sets bootstrap as in Lee et al. 2022 (Experiment
// Setup); this is that subsystem for the library's chains, after Cheon, Han,
// Kim, Kim and Song 2018 with a polynomial for the modular reduction:
//
// * ModRaise: a level-0 ciphertext read over the chain up to `level`; it
//   decrypts to t = m + q0 I, I a small integer polynomial (|I| <= K with
//   high probability for a sparse secret).
// * CoeffToSlot: slots z = U w, w = (t_lo + i t_hi) / Delta the N/2 complex
//   coefficients, U the decoding map. U = F_(log n) ... F_1 BR (radix-2
//   decimation in time, stage s pairing slots p and p + h, h = 2^(s-1):
//   out[p] = x[p] + w_r x[p + h], out[p + h] = x[p] - w_r x[p + h], r = p mod
//   2h, w_r = exp(2 pi i (5^r mod 8h) / 8h)). The stages' inverses (without
//   their halvings), merged into a few levels of 2^(r+1) - 1 cyclic
//   diagonals, give n BR(w); the conjugation X -> X^(2N-1) splits real and
//   imaginary parts (the latter times -i = X^(3N/2)), and the constant
//   2^-(e + log2 N), applied as a wide integer over two rescales, gives
//   y = t / (Delta 2^e) in [-1, 1], 2^e >= (K + 1) q0 / Delta.
// * EvalMod: sum_j a_j T_j(y), the Chebyshev interpolant of
//   (c / 2 pi) sin(2 pi 2^e y / c), c = q0 / Delta, which is m / Delta.
// * SlotToCoeff: m_lo + i m_hi (i = X^(N/2)), then the merged F stages.
//
// A linear transform is z -> sum_k d_k (.) rot(z, base + k stride), applied by
// baby-step giant-step: one hoisted ModUp for the baby rotations j stride
// (j < g1), per giant step the products with the diagonals pre-rotated by
// -(base + g1 i stride) accumulated, rescaled once and rotated by
// base + g1 i stride; with double hoisting the baby rotations stay in QP_l
// and each giant step's products are summed over QP_l and divided by P q_l
// once. Its plaintexts are encoded once, at creation, for the level and
// input scale it is applied at.
#include <math.h>

#include <algorithm>
#include <complex>
#include <map>

#include "modarith.cuh"
#include "ops.h"

namespace ck {

namespace {

constexpr int TPB = 256;
inline unsigned grid_for(size_t total) {
  size_t g = (total + TPB - 1) / TPB;
  const size_t cap = 152 * 32;
  return (unsigned)(g < cap ? (g ? g : 1) : cap);
}
#define GRID_LOOP(idx, total) \
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (total); idx += (size_t)gridDim.x * blockDim.x)

// centred int64 of residues mod q0
__global__ void centre_kernel(const uint64_t* x, int64_t* v, size_t total, uint64_t q0) {
  GRID_LOOP(i, total) {
    const uint64_t a = x[i];
    v[i] = a > q0 / 2 ? -(int64_t)(q0 - a) : (int64_t)a;
  }
}

// pt[t] = X^pos (neg: -X^pos) mod q_t, coefficient form
__global__ void monomial_kernel(uint64_t* pt, int l, int log_n, size_t pos, int neg,
                                const Mod* mods) {
  const size_t N = (size_t)1 << log_n;
  GRID_LOOP(i, (size_t)l * N) {
    const int t = (int)(i >> log_n);
    pt[i] = (i & (N - 1)) == pos ? (neg ? mods[t].q - 1 : 1) : 0;
  }
}

// residue mod q of the integer value of a double (|v| < 2^1023, integral)
uint64_t double_residue(double v, uint64_t q) {
  const bool neg = v < 0;
  const double a = fabs(v);
  uint64_t r;
  if (a < 9007199254740992.0) {  // 2^53: exact in uint64
    r = (uint64_t)a % q;
  } else {
    int ex;
    const double fr = frexp(a, &ex);  // a = fr 2^ex, fr in [0.5, 1)
    const uint64_t mant = (uint64_t)ldexp(fr, 53);
    r = mulmod_h(mant % q, powmod_h(2, (uint64_t)(ex - 53), q), q);
  }
  return neg && r ? q - r : r;
}

}  // namespace

Ct op_mod_raise(Ctx& c, const ckks_ct& a, int level) {
  if (a.level != 0) throw Error(CKKS_ERR_LEVEL, "ModRaise takes a level-0 ciphertext");
  if (level < 0 || level > c.L) throw Error(CKKS_ERR_LEVEL, "level out of range");
  const size_t polys = a.B * 2, N = c.N;
  DevBuf x(&c, polys * N * 8), v(&c, polys * N * 8);
  CK_CUDA(cudaMemcpyAsync(x.p, a.d.p, polys * N * 8, cudaMemcpyDeviceToDevice, c.stream));
  ntt_inverse(c, x.u64(), polys, c.iota(), 1);
  {
  Launch L_(c, K_INT_RNS, 2.0 * polys * N * 8);
  centre_kernel<<<grid_for(polys * N), TPB, 0, c.stream>>>(x.u64(), static_cast<int64_t*>(v.p),
                                                           polys * N, c.mod[0]);
  CK_CUDA(cudaGetLastError());
  }
  Ct r = ct_alloc(c, a.B, level, a.scale);
  k_int_to_rns(c, static_cast<int64_t*>(v.p), r->d.u64(), polys, level + 1, c.iota());
  ntt_forward(c, r->d.u64(), polys * (level + 1), c.iota(), level + 1);
  return r;
}

Ct op_mul_monomial(Ctx& c, const ckks_ct& a, int64_t k) {
  const int64_t M = 2 * (int64_t)c.N;
  k = ((k % M) + M) % M;
  const int l = a.level + 1;
  DevBuf pt(&c, (size_t)l * c.N * 8);
  {
  Launch L_(c, K_COPY, (double)l * c.N * 8);
  monomial_kernel<<<grid_for((size_t)l * c.N), TPB, 0, c.stream>>>(
      pt.u64(), l, c.log_n, (size_t)(k % (int64_t)c.N), k >= (int64_t)c.N, c.dmod());
  CK_CUDA(cudaGetLastError());
  }
  ntt_forward(c, pt.u64(), l, c.iota(), l);
  Ct r = ct_alloc(c, a.B, a.level, a.scale);
  k_mul_pt(c, a.d.u64(), pt.u64(), r->d.u64(), a.B * 2 * l, l);
  return r;
}

Ct op_conjugate(Ctx& c, const ckks_keys& keys, const ckks_ct& a) {
  auto v = op_galois_many(c, keys, a, {2 * c.N - 1});
  return std::move(v[0]);
}

// a * cst for a constant far below 1, landing on the canonical scale of
// level - 2: the integer rint(cst S2), S2 = Delta_(l-2) q_l q_(l-1) / scale,
// applied by its residues (however large), then two rescales
Ct op_mul_const_wide(Ctx& c, const ckks_ct& a, double cst) {
  const int lv = a.level;
  if (lv < 2) throw Error(CKKS_ERR_LEVEL, "level exhausted");
  const double S2 = c.delta[lv - 2] * (double)c.mod[lv] * (double)c.mod[lv - 1] / a.scale;
  const double kv = rint(cst * S2);
  if (!(fabs(kv) < 1e300)) throw Error(CKKS_ERR_OVERFLOW, "constant does not fit");
  std::vector<uint64_t> res(lv + 1);
  for (int t = 0; t <= lv; t++) res[t] = double_residue(kv, c.mod[t]);
  Ct t = ct_alloc(c, a.B, lv, a.scale * S2);
  k_mul_limbs(c, a.d.u64(), res, t->d.u64(), a.B * 2 * (lv + 1), lv + 1);
  Ct once = op_rescale(c, *t);
  return op_rescale(c, *once);
}

}  // namespace ck

// ---------------------------------------------------------------- handles
struct ckks_lt {
  ck::Ctx* ctx;
  int level;
  double in_scale, pt_scale;
  int64_t base, stride;
  int n_diag, g1, g2;
  int form;               // 0: hoisted baby steps; 1: double hoisting (QP_l)
  std::vector<int> slot;  // [n_diag]: plaintext index, -1 = zero diagonal
  ck::DevBuf pts;         // [nonzero][rows][N], rows = level + 1 (+ alpha if form 1)
};

struct ckks_boot {
  ck::Ctx* ctx;
  int e;
  std::vector<double> cheb;
  std::vector<const ckks_lt*> cts, stc;
  std::vector<std::unique_ptr<ckks_lt>> owned;
};

namespace ck {

namespace {

int default_g1(int K) {
  int g = 1;
  while ((int64_t)g * g < K) g *= 2;
  return g;
}

int64_t mod_n(int64_t x, int64_t n) { return ((x % n) + n) % n; }

}  // namespace

std::unique_ptr<ckks_lt> lt_create(Ctx& c, int level, double in_scale, int64_t base,
                                   int64_t stride, int n_diag, const double* re, const double* im,
                                   int g1, int form) {
  if (level < 1 || level > c.L) throw Error(CKKS_ERR_LEVEL, "level out of range");
  if (n_diag < 1 || !re || !im) throw Error(CKKS_ERR_INVALID_ARG, "no diagonals");
  if (g1 < 0) throw Error(CKKS_ERR_INVALID_ARG, "negative baby-step count");
  if (form != 0 && form != 1) throw Error(CKKS_ERR_INVALID_ARG, "unknown transform form");
  const int64_t n = (int64_t)c.N / 2;
  auto lt = std::make_unique<ckks_lt>();
  lt->ctx = &c;
  lt->level = level;
  lt->in_scale = in_scale > 0 ? in_scale : c.delta[level];
  lt->pt_scale = plain_scale(c, lt->in_scale, level);
  lt->base = base;
  lt->stride = stride;
  lt->n_diag = n_diag;
  // a double-hoisted baby step is a key product only (no ModDown) while a
  // giant step is a whole rotation: twice the square-root rule's baby steps
  // measured fastest for the refresh's levels (63 diagonals: 16 against 8)
  lt->g1 = g1 ? g1 : (form == 1 ? default_g1(4 * n_diag) : default_g1(n_diag));
  lt->g2 = (n_diag + lt->g1 - 1) / lt->g1;
  lt->form = form;
  // pre-rotate the nonzero diagonals by -(base + g1 i stride): np.roll(d, G)
  std::vector<double> hr, hi;
  int nz = 0;
  lt->slot.assign(n_diag, -1);
  for (int k = 0; k < n_diag; k++) {
    const double* dr = re + (size_t)k * n;
    const double* di = im + (size_t)k * n;
    bool any = false;
    for (int64_t p = 0; p < n && !any; p++) any = dr[p] != 0.0 || di[p] != 0.0;
    if (!any) continue;
    const int64_t G = base + (int64_t)lt->g1 * (k / lt->g1) * stride;
    lt->slot[k] = nz++;
    for (int64_t p = 0; p < n; p++) {
      const int64_t src = mod_n(p - G, n);
      hr.push_back(dr[src]);
      hi.push_back(di[src]);
    }
  }
  ConvTables& T = c.tables(level);
  const int rows = form == 1 ? T.rows : level + 1;
  const int16_t* pattern = form == 1 ? static_cast<const int16_t*>(T.qp_pattern.p) : c.iota();
  lt->pts = DevBuf(&c, std::max<size_t>((size_t)nz * rows * c.N * 8, 8));
  if (nz) {
    DevBuf dr(&c, hr.size() * 8), di(&c, hi.size() * 8);
    CK_CUDA(cudaMemcpyAsync(dr.p, hr.data(), hr.size() * 8, cudaMemcpyHostToDevice, c.stream));
    CK_CUDA(cudaMemcpyAsync(di.p, hi.data(), hi.size() * 8, cudaMemcpyHostToDevice, c.stream));
    const int rc = encode_rows(c, static_cast<const double*>(dr.p), nz, n, rows, pattern,
                               lt->pt_scale, lt->pts.u64(), static_cast<const double*>(di.p));
    if (rc != CKKS_OK) throw Error(rc, "diagonal does not fit its scale");
  }
  CK_CUDA(cudaStreamSynchronize(c.stream));
  return lt;
}

std::vector<int64_t> lt_steps(const Ctx& c, const ckks_lt& lt) {
  const int64_t n = (int64_t)c.N / 2;
  std::vector<int64_t> st;
  for (int j = 1; j < lt.g1; j++) st.push_back(mod_n(j * lt.stride, n));
  for (int i = 0; i < lt.g2; i++) st.push_back(mod_n(lt.base + (int64_t)lt.g1 * i * lt.stride, n));
  std::sort(st.begin(), st.end());
  st.erase(std::unique(st.begin(), st.end()), st.end());
  if (!st.empty() && st[0] == 0) st.erase(st.begin());
  return st;
}

// double hoisting: baby rotations kept in QP_l (R_0 = P v, R_j the key
// product of sigma_j(ModUp(c1)) plus P sigma_j(c0)), each giant step's
// products summed over QP_l and divided by P q_l once
Ct lt_apply_double(Ctx& c, const ckks_keys& keys, const ckks_lt& lt, const ckks_ct& v) {
  const int64_t n = (int64_t)c.N / 2;
  const int lv = v.level, l = lv + 1;
  ConvTables& T = c.tables(lv);
  const size_t qp_words = v.B * 2 * (size_t)T.rows * c.N;
  std::vector<DevBuf> R;
  R.emplace_back(&c, qp_words * 8);
  k_qp_lift(c, v.d.u64(), v.B, lv, nullptr, R[0].u64());
  DevBuf ext;
  for (int j = 1; j < lt.g1; j++) {
    const uint64_t g = c.galois(j * lt.stride);
    DevBuf kt;
    const uint64_t* key = switch_key_words(c, keys, g, kt);
    if (!ext.p) {
      ext = DevBuf(&c, v.B * T.beta * T.rows * c.N * 8);
      modup(c, v.d.u64() + (size_t)l * c.N, v.B, lv, ext.u64(), 2 * (size_t)l * c.N);
    }
    DevBuf acc = keyswitch_qp(c, ext.u64(), v.B, lv, key, g);
    k_qp_lift(c, v.d.u64(), v.B, lv, c.perm(g), acc.u64());
    R.push_back(std::move(acc));
  }
  ext.reset();
  double s = v.scale * lt.pt_scale / (double)c.mod[lv];
  if (fabs(s / c.delta[lv - 1] - 1.0) < SNAP) s = c.delta[lv - 1];
  Ct z;
  DevBuf acc(&c, qp_words * 8);
  for (int i = 0; i < lt.g2; i++) {
    const int64_t G = lt.base + (int64_t)lt.g1 * i * lt.stride;
    std::vector<const uint64_t*> as, ps;
    for (int j = 0; j < lt.g1; j++) {
      const int k = lt.g1 * i + j;
      if (k >= lt.n_diag || lt.slot[k] < 0) continue;
      as.push_back(R[j].u64());
      ps.push_back(lt.pts.u64() + (size_t)lt.slot[k] * T.rows * c.N);
    }
    if (as.empty()) continue;
    k_mul_pt_sum(c, as, ps, acc.u64(), v.B * 2, T.rows, static_cast<const int16_t*>(T.qp_pattern.p),
                 true);
    Ct inner = ct_alloc(c, v.B, lv - 1, s);
    div_p_ql(c, acc.u64(), v.B, lv, inner->d.u64());
    if (mod_n(G, n)) inner = op_rotate(c, keys, *inner, mod_n(G, n));
    z = z ? op_add(c, *z, *inner, false) : std::move(inner);
  }
  if (!z) throw Error(CKKS_ERR_INVALID_ARG, "transform with only zero diagonals");
  return z;
}

Ct lt_apply(Ctx& c, const ckks_keys& keys, const ckks_lt& lt, const ckks_ct& v) {
  if (v.level != lt.level) throw Error(CKKS_ERR_LEVEL, "transform built for another level");
  if (fabs(v.scale / lt.in_scale - 1.0) > SNAP) throw Error(CKKS_ERR_SCALE, "transform built for another scale");
  if (lt.form == 1) return lt_apply_double(c, keys, lt, v);
  const int64_t n = (int64_t)c.N / 2;
  const int l = v.level + 1;
  std::vector<int64_t> bsteps;
  for (int j = 0; j < lt.g1; j++) bsteps.push_back(j * lt.stride);
  std::vector<Ct> baby = op_rotate_many(c, keys, v, bsteps);
  Ct z;
  for (int i = 0; i < lt.g2; i++) {
    const int64_t G = lt.base + (int64_t)lt.g1 * i * lt.stride;
    std::vector<const uint64_t*> as, ps;
    for (int j = 0; j < lt.g1; j++) {
      const int k = lt.g1 * i + j;
      if (k >= lt.n_diag || lt.slot[k] < 0) continue;
      as.push_back(baby[j]->d.u64());
      ps.push_back(lt.pts.u64() + (size_t)lt.slot[k] * l * c.N);
    }
    if (as.empty()) continue;
    Ct acc = ct_alloc(c, v.B, v.level, v.scale * lt.pt_scale);
    k_mul_pt_sum(c, as, ps, acc->d.u64(), v.B * 2, l, c.iota(), true);
    Ct inner = op_rescale(c, *acc);
    if (mod_n(G, n)) inner = op_rotate(c, keys, *inner, mod_n(G, n));
    z = z ? op_add(c, *z, *inner, false) : std::move(inner);
  }
  if (!z) throw Error(CKKS_ERR_INVALID_ARG, "transform with only zero diagonals");
  return z;
}

void boot_coeff_to_slot(Ctx& c, const ckks_keys& keys, const ckks_boot& b, const ckks_ct& raised,
                        Ct& lo, Ct& hi) {
  Ct ct;
  const ckks_ct* cur = &raised;
  for (const ckks_lt* lt : b.cts) {
    ct = lt_apply(c, keys, *lt, *cur);
    cur = ct.get();
  }
  Ct cj = op_conjugate(c, keys, *cur);
  Ct re2 = op_add(c, *cur, *cj, false);
  Ct im2 = op_mul_monomial(c, *op_add(c, *cur, *cj, true), 3 * (int64_t)c.N / 2);
  const double f = ldexp(1.0, -(b.e + c.log_n));
  lo = op_mul_const_wide(c, *re2, f);
  hi = op_mul_const_wide(c, *im2, f);
}

Ct boot_slot_to_coeff(Ctx& c, const ckks_keys& keys, const ckks_boot& b, const ckks_ct& lo,
                      const ckks_ct& hi) {
  const int lv = std::min(lo.level, hi.level);
  Ct l2 = op_level_down(c, lo, lv), h2 = op_level_down(c, hi, lv);
  Ct ct = op_add(c, *l2, *op_mul_monomial(c, *h2, (int64_t)c.N / 2), false);
  for (const ckks_lt* lt : b.stc) ct = lt_apply(c, keys, *lt, *ct);
  return ct;
}

Ct bootstrap(Ctx& c, const ckks_keys& keys, const ckks_boot& b, const ckks_ct& in) {
  Ct raised = op_mod_raise(c, in, b.cts.empty() ? c.L : b.cts[0]->level);
  Ct lo, hi;
  boot_coeff_to_slot(c, keys, b, *raised, lo, hi);
  raised.reset();
  // both halves through EvalMod as one batch of 2B (every step is per element)
  Ct both = op_concat(c, {lo.get(), hi.get()});
  lo.reset();
  hi.reset();
  Ct m = cheb_eval(c, keys, *both, b.cheb);
  both.reset();
  const size_t half = m->words() / 2;
  Ct mlo = ct_alloc(c, in.B, m->level, m->scale), mhi = ct_alloc(c, in.B, m->level, m->scale);
  CK_CUDA(cudaMemcpyAsync(mlo->d.p, m->d.p, half * 8, cudaMemcpyDeviceToDevice, c.stream));
  CK_CUDA(cudaMemcpyAsync(mhi->d.p, m->d.u64() + half, half * 8, cudaMemcpyDeviceToDevice,
                          c.stream));
  m.reset();
  return boot_slot_to_coeff(c, keys, b, *mlo, *mhi);
}

// A batch refreshed with one bootstrap per S / nb ciphertexts (nb the least
// power of two >= n_out): each ciphertext masked to its slots [0, n_out)
// (one level), packed by a rotation tree (ciphertext b at slots b nb..),
// brought to level 0 and bootstrapped, unpacked by a rotation tree
// (u_(x + s) = rot(u_x, s nb) for s = top/2 .. 1); the unpacked ciphertexts
// hold the others' blocks beyond [0, n_out), which the next layer's input
// mask removes.
Ct refresh_packed(Ctx& c, const ckks_keys& keys, const ckks_boot& b, const ckks_ct& in,
                  int n_out) {
  if (in.level < 1) throw Error(CKKS_ERR_LEVEL, "packing needs one level");
  const size_t S = c.N / 2;
  size_t nb = 1;
  while (nb < (size_t)n_out) nb *= 2;
  if (nb > S) throw Error(CKKS_ERR_INVALID_ARG, "block larger than the slots");
  const size_t per = S / nb;
  std::vector<double> mask((size_t)n_out, 1.0);
  const double Spt = plain_scale(c, in.scale, in.level);
  DevBuf pt = encode_vec(c, mask.data(), mask.size(), in.level, Spt);
  Ct masked = op_mul_pt(c, in, pt.u64(), Spt);
  const size_t words = masked->words() / masked->B;
  std::vector<Ct> outs;
  for (size_t g = 0; g < in.B; g += per) {
    const size_t cnt = std::min(per, in.B - g);
    std::vector<Ct> cur;
    for (size_t k = 0; k < cnt; k++) {
      Ct one = ct_alloc(c, 1, masked->level, masked->scale);
      CK_CUDA(cudaMemcpyAsync(one->d.p, masked->d.u64() + (g + k) * words, words * 8,
                              cudaMemcpyDeviceToDevice, c.stream));
      cur.push_back(std::move(one));
    }
    int64_t step = (int64_t)nb;
    while (cur.size() > 1) {
      std::vector<Ct> nxt;
      for (size_t k = 0; k < cur.size(); k += 2) {
        if (k + 1 < cur.size())
          nxt.push_back(op_add(c, *cur[k], *op_rotate(c, keys, *cur[k + 1], -step), false));
        else
          nxt.push_back(std::move(cur[k]));
      }
      cur = std::move(nxt);
      step *= 2;
    }
    Ct fresh = bootstrap(c, keys, b, *op_level_down(c, *cur[0], 0));
    std::map<size_t, Ct> u;
    u[0] = std::move(fresh);
    size_t s = 0;
    if (cnt > 1) {
      s = 1;
      while (2 * s <= cnt - 1) s *= 2;
    }
    for (; s >= 1; s /= 2) {
      std::vector<size_t> have;
      for (auto& kv : u) have.push_back(kv.first);
      for (size_t x : have)
        if (x + s < cnt && !u.count(x + s)) u[x + s] = op_rotate(c, keys, *u[x], (int64_t)(s * nb));
    }
    for (size_t k = 0; k < cnt; k++) outs.push_back(std::move(u[k]));
  }
  if (outs.size() == 1) return std::move(outs[0]);
  std::vector<const ckks_ct*> parts;
  for (auto& o : outs) parts.push_back(o.get());
  return op_concat(c, parts);
}

// ---------------------------------------------------------------- the plan
namespace {

using cd = std::complex<double>;
using Diags = std::map<int64_t, std::vector<cd>>;

std::vector<cd> stage_roots(int64_t h) {
  std::vector<cd> w(h);
  for (int64_t r = 0; r < h; r++) {
    const double e = (double)powmod_h(5, (uint64_t)r, 8 * (uint64_t)h);
    const double ang = 2.0 * M_PI * e / (8.0 * (double)h);
    w[r] = cd(cos(ang), sin(ang));
  }
  return w;
}

// {offset mod n: diagonal} of F_s, or of 2 F_s^-1
Diags fft_stage(int64_t n, int s, bool inverse) {
  const int64_t h = (int64_t)1 << (s - 1);
  const std::vector<cd> w = stage_roots(h);
  std::vector<cd> d0(n), dp(n), dm(n);
  for (int64_t p = 0; p < n; p++) {
    const int64_t r = p % (2 * h);
    const bool lower = r < h;
    const cd wr = w[lower ? r : r - h];
    if (!inverse) {
      d0[p] = lower ? cd(1, 0) : -wr;
      dp[p] = lower ? wr : cd(0, 0);
      dm[p] = lower ? cd(0, 0) : cd(1, 0);
    } else {
      d0[p] = lower ? cd(1, 0) : -std::conj(wr);
      dp[p] = lower ? cd(1, 0) : cd(0, 0);
      dm[p] = lower ? cd(0, 0) : std::conj(wr);
    }
  }
  Diags d;
  auto put = [&](int64_t o, std::vector<cd>& v) {
    o = mod_n(o, n);
    auto it = d.find(o);
    if (it == d.end()) {
      d[o] = v;
    } else {
      for (int64_t p = 0; p < n; p++) it->second[p] += v[p];
    }
  };
  put(0, d0);
  put(h, dp);
  put(-h, dm);
  return d;
}

// (A B)_o = sum over a + b = o of A_a (.) rot(B_b, a)
Diags compose(int64_t n, const Diags& A, const Diags& B) {
  Diags out;
  for (const auto& a : A) {
    for (const auto& b : B) {
      const int64_t o = mod_n(a.first + b.first, n);
      auto it = out.find(o);
      if (it == out.end()) it = out.emplace(o, std::vector<cd>(n)).first;
      for (int64_t p = 0; p < n; p++) {
        it->second[p] += a.second[p] * b.second[mod_n(p + a.first, n)];
      }
    }
  }
  return out;
}

}  // namespace

// The merged levels of U's factors (SlotToCoeff: F_1 .. F_(log n);
// CoeffToSlot: 2 F_(log n)^-1 .. 2 F_1^-1), n_levels groups of consecutive
// stages; a group with h = 2^a .. 2^(a+r-1) has offsets k 2^a, |k| < 2^r.
// Writes for each level: base, stride, n_diag, and the diagonals.
void boot_levels(const Ctx& c, int n_levels, bool inverse, std::vector<int64_t>& base,
                 std::vector<int64_t>& stride, std::vector<std::vector<double>>& re,
                 std::vector<std::vector<double>>& im) {
  const int64_t n = (int64_t)c.N / 2;
  const int log_n = c.log_n - 1;
  if (n_levels < 1 || n_levels > log_n) throw Error(CKKS_ERR_INVALID_ARG, "transform levels out of range");
  std::vector<int> stages;
  for (int s = 1; s <= log_n; s++) stages.push_back(inverse ? log_n + 1 - s : s);
  size_t k0 = 0;
  for (int g = 0; g < n_levels; g++) {
    const int sz = log_n / n_levels + (g < log_n % n_levels ? 1 : 0);
    std::vector<int> grp(stages.begin() + k0, stages.begin() + k0 + sz);
    k0 += sz;
    Diags M;
    bool first = true;
    for (int s : grp) {
      Diags st = fft_stage(n, s, inverse);
      M = first ? st : compose(n, st, M);
      first = false;
    }
    const int a = *std::min_element(grp.begin(), grp.end()) - 1;
    const int64_t str = (int64_t)1 << a, span = ((int64_t)1 << sz) - 1;
    base.push_back(-span * str);
    stride.push_back(str);
    std::vector<double> r, i;
    std::map<int64_t, bool> seen;
    for (int64_t k = 0; k < 2 * span + 1; k++) {
      const int64_t o = mod_n(-span * str + k * str, n);
      auto it = M.find(o);
      const bool use = it != M.end() && !seen.count(o);
      for (int64_t p = 0; p < n; p++) {
        r.push_back(use ? it->second[p].real() : 0.0);
        i.push_back(use ? it->second[p].imag() : 0.0);
      }
      if (use) seen[o] = true;
    }
    re.push_back(std::move(r));
    im.push_back(std::move(i));
  }
}

int boot_exponent(const Ctx& c, int K) {
  return (int)ceil(log2((K + 1) * ((double)c.mod[0] / c.delta[0])));
}

// Chebyshev coefficients of the interpolant of (c / 2 pi) sin(2 pi 2^e y / c)
// at the degree + 1 Chebyshev points of the first kind
std::vector<double> boot_cheb(const Ctx& c, int e, int degree) {
  const double cq = (double)c.mod[0] / c.delta[0];
  const double w = 2.0 * M_PI * ldexp(1.0, e) / cq;
  const int m = degree + 1;
  std::vector<double> x(m), f(m), a(m, 0.0);
  for (int k = 0; k < m; k++) {
    x[k] = -cos(M_PI * (k + 0.5) / m);
    f[k] = cq / (2.0 * M_PI) * sin(w * x[k]);
  }
  for (int k = 0; k < m; k++) {  // a_j = sum_k f(x_k) T_j(x_k) (then normalised)
    double t0 = 1.0, t1 = x[k];
    a[0] += f[k];
    if (m > 1) a[1] += f[k] * x[k];
    for (int j = 2; j < m; j++) {
      const double t2 = 2.0 * x[k] * t1 - t0;
      a[j] += f[k] * t2;
      t0 = t1;
      t1 = t2;
    }
  }
  a[0] /= m;
  for (int j = 1; j < m; j++) a[j] /= 0.5 * m;
  return a;
}

}  // namespace ck

using namespace ck;

namespace {
template <class F>
int guard(F&& f) {
  try {
    f();
    return CKKS_OK;
  } catch (...) {
    return api_error();
  }
}
void need(bool cond, const char* what) {
  if (!cond) throw Error(CKKS_ERR_INVALID_ARG, what);
}
}  // namespace

extern "C" {

int ckks_keygen_ex(ckks_ctx* ctx, uint64_t seed, int hamming_weight, const int32_t* rot_steps,
                   size_t n_steps, int conjugation, uint64_t public_seed, ckks_keys** out) {
  return guard([&] {
    need(ctx && out, "NULL argument");
    need(n_steps == 0 || rot_steps, "rot_steps is NULL");
    need(hamming_weight >= 0, "negative Hamming weight");
    need(public_seed == 0 || public_seed != seed, "the public seed must differ from the seed");
    std::vector<int64_t> steps(rot_steps, rot_steps + n_steps);
    *out = keygen(ctx->c, seed, steps, hamming_weight, conjugation != 0, public_seed).release();
  });
}

int ckks_mod_raise(ckks_ctx* ctx, const ckks_ct* in, int level, ckks_ct** out) {
  return guard([&] {
    need(ctx && in && out, "NULL argument");
    *out = op_mod_raise(ctx->c, *in, level).release();
  });
}

int ckks_conjugate(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* in, ckks_ct** out) {
  return guard([&] {
    need(ctx && keys && in && out, "NULL argument");
    *out = op_conjugate(ctx->c, *keys, *in).release();
  });
}

int ckks_mul_monomial(ckks_ctx* ctx, const ckks_ct* in, int64_t k, ckks_ct** out) {
  return guard([&] {
    need(ctx && in && out, "NULL argument");
    *out = op_mul_monomial(ctx->c, *in, k).release();
  });
}

int ckks_mul_const_wide(ckks_ctx* ctx, const ckks_ct* in, double value, ckks_ct** out) {
  return guard([&] {
    need(ctx && in && out, "NULL argument");
    *out = op_mul_const_wide(ctx->c, *in, value).release();
  });
}

int ckks_lt_create(ckks_ctx* ctx, int level, double in_scale, int64_t base, int64_t stride,
                   size_t n_diag, const double* re, const double* im, int g1, int form,
                   ckks_lt** out) {
  return guard([&] {
    need(ctx && re && im && out, "NULL argument");
    need(n_diag >= 1 && n_diag <= ctx->c.N, "diagonal count out of range");
    *out = lt_create(ctx->c, level, in_scale, base, stride, (int)n_diag, re, im, g1, form)
               .release();
  });
}

int ckks_lt_destroy(ckks_lt* lt) {
  return guard([&] { delete lt; });
}

int ckks_lt_rotations(const ckks_lt* lt, int32_t* steps, size_t cap, size_t* n) {
  return guard([&] {
    need(lt && n, "NULL argument");
    auto st = lt_steps(*lt->ctx, *lt);
    *n = st.size();
    need(cap == 0 || steps, "steps is NULL");
    for (size_t i = 0; i < st.size() && i < cap; i++) steps[i] = (int32_t)st[i];
  });
}

int ckks_lt_apply(ckks_ctx* ctx, const ckks_keys* keys, const ckks_lt* lt, const ckks_ct* in,
                  ckks_ct** out) {
  return guard([&] {
    need(ctx && keys && lt && in && out, "NULL argument");
    need(lt->ctx == &ctx->c, "transform of another context");
    *out = lt_apply(ctx->c, *keys, *lt, *in).release();
  });
}

int ckks_boot_create(ckks_ctx* ctx, int K, int degree, int cts_levels, int stc_levels, int form,
                     ckks_boot** out) {
  return guard([&] {
    need(ctx && out, "NULL argument");
    need(K >= 1 && degree >= 1, "K and degree must be positive");
    Ctx& c = ctx->c;
    auto b = std::make_unique<ckks_boot>();
    b->ctx = &c;
    b->e = boot_exponent(c, K);
    b->cheb = boot_cheb(c, b->e, degree);
    const int64_t n = (int64_t)c.N / 2;
    int level = c.L;
    for (int pass = 0; pass < 2; pass++) {
      const bool inverse = pass == 0;
      std::vector<int64_t> base, stride;
      std::vector<std::vector<double>> re, im;
      boot_levels(c, inverse ? cts_levels : stc_levels, inverse, base, stride, re, im);
      if (!inverse) level = level - 2 - cheb_levels(degree);
      for (size_t g = 0; g < base.size(); g++) {
        const double in_scale = inverse && g == 0 ? c.delta[0] : c.delta[level];
        auto lt = lt_create(c, level, in_scale, base[g], stride[g], (int)(re[g].size() / n),
                            re[g].data(), im[g].data(), 0, form);
        (inverse ? b->cts : b->stc).push_back(lt.get());
        b->owned.push_back(std::move(lt));
        level -= 1;
      }
    }
    if (level < 0) throw Error(CKKS_ERR_LEVEL, "the chain is too short for this bootstrapping");
    *out = b.release();
  });
}

int ckks_boot_create_ex(ckks_ctx* ctx, int e, const double* cheb, size_t n_cheb,
                        const ckks_lt* const* cts, size_t n_cts, const ckks_lt* const* stc,
                        size_t n_stc, ckks_boot** out) {
  return guard([&] {
    need(ctx && cheb && out && (cts || !n_cts) && (stc || !n_stc), "NULL argument");
    need(n_cheb >= 2 && n_cts >= 1 && n_stc >= 1, "empty plan");
    auto b = std::make_unique<ckks_boot>();
    b->ctx = &ctx->c;
    b->e = e;
    b->cheb.assign(cheb, cheb + n_cheb);
    for (size_t i = 0; i < n_cts; i++) {
      need(cts[i] && cts[i]->ctx == &ctx->c, "transform of another context");
      b->cts.push_back(cts[i]);
    }
    for (size_t i = 0; i < n_stc; i++) {
      need(stc[i] && stc[i]->ctx == &ctx->c, "transform of another context");
      b->stc.push_back(stc[i]);
    }
    *out = b.release();
  });
}

int ckks_boot_destroy(ckks_boot* boot) {
  return guard([&] { delete boot; });
}

int ckks_boot_info(const ckks_boot* boot, int* e, int* cts_level, int* stc_level,
                   size_t* n_cheb) {
  return guard([&] {
    need(boot, "NULL argument");
    if (e) *e = boot->e;
    if (cts_level) *cts_level = boot->cts[0]->level;
    if (stc_level) *stc_level = boot->stc[0]->level;
    if (n_cheb) *n_cheb = boot->cheb.size();
  });
}

int ckks_boot_coefficients(const ckks_boot* boot, double* cheb, size_t cap) {
  return guard([&] {
    need(boot && cheb, "NULL argument");
    need(cap >= boot->cheb.size(), "buffer too small");
    std::copy(boot->cheb.begin(), boot->cheb.end(), cheb);
  });
}

int ckks_boot_diagonals(const ckks_boot* boot, int inverse, size_t index, int64_t* base,
                        int64_t* stride, size_t* n_diag) {
  return guard([&] {
    need(boot && base && stride && n_diag, "NULL argument");
    const auto& v = inverse ? boot->cts : boot->stc;
    need(index < v.size(), "transform index out of range");
    *base = v[index]->base;
    *stride = v[index]->stride;
    *n_diag = (size_t)v[index]->n_diag;
  });
}

int ckks_boot_levels(ckks_ctx* ctx, int n_levels, int inverse, size_t index, double* re,
                     double* im, size_t cap, int64_t* base, int64_t* stride, size_t* n_diag) {
  return guard([&] {
    need(ctx && base && stride && n_diag, "NULL argument");
    std::vector<int64_t> b, s;
    std::vector<std::vector<double>> r, i;
    boot_levels(ctx->c, n_levels, inverse != 0, b, s, r, i);
    need(index < b.size(), "level index out of range");
    const size_t n = ctx->c.N / 2;
    *base = b[index];
    *stride = s[index];
    *n_diag = r[index].size() / n;
    if (re || im) {
      need(re && im && cap >= r[index].size(), "buffer too small");
      std::copy(r[index].begin(), r[index].end(), re);
      std::copy(i[index].begin(), i[index].end(), im);
    }
  });
}

int ckks_boot_rotations(const ckks_boot* boot, int32_t* steps, size_t cap, size_t* n) {
  return guard([&] {
    need(boot && n, "NULL argument");
    std::vector<int64_t> all;
    for (const auto* v : {&boot->cts, &boot->stc})
      for (const ckks_lt* lt : *v) {
        auto st = lt_steps(*boot->ctx, *lt);
        all.insert(all.end(), st.begin(), st.end());
      }
    std::sort(all.begin(), all.end());
    all.erase(std::unique(all.begin(), all.end()), all.end());
    *n = all.size();
    need(cap == 0 || steps, "steps is NULL");
    for (size_t i = 0; i < all.size() && i < cap; i++) steps[i] = (int32_t)all[i];
  });
}

int ckks_boot_coeff_to_slot(ckks_ctx* ctx, const ckks_keys* keys, const ckks_boot* boot,
                            const ckks_ct* raised, ckks_ct** lo, ckks_ct** hi) {
  return guard([&] {
    need(ctx && keys && boot && raised && lo && hi, "NULL argument");
    Ct l, h;
    boot_coeff_to_slot(ctx->c, *keys, *boot, *raised, l, h);
    *lo = l.release();
    *hi = h.release();
  });
}

int ckks_boot_eval_mod(ckks_ctx* ctx, const ckks_keys* keys, const ckks_boot* boot,
                       const ckks_ct* in, ckks_ct** out) {
  return guard([&] {
    need(ctx && keys && boot && in && out, "NULL argument");
    *out = cheb_eval(ctx->c, *keys, *in, boot->cheb).release();
  });
}

int ckks_boot_slot_to_coeff(ckks_ctx* ctx, const ckks_keys* keys, const ckks_boot* boot,
                            const ckks_ct* lo, const ckks_ct* hi, ckks_ct** out) {
  return guard([&] {
    need(ctx && keys && boot && lo && hi && out, "NULL argument");
    *out = boot_slot_to_coeff(ctx->c, *keys, *boot, *lo, *hi).release();
  });
}

int ckks_bootstrap(ckks_ctx* ctx, const ckks_keys* keys, const ckks_boot* boot,
                   const ckks_ct* in, ckks_ct** out) {
  return guard([&] {
    need(ctx && keys && boot && in && out, "NULL argument");
    need(boot->ctx == &ctx->c, "plan of another context");
    *out = bootstrap(ctx->c, *keys, *boot, *in).release();
  });
}

}  // extern "C"
