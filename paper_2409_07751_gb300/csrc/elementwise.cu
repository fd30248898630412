// Elementwise kernels over ciphertext batches laid out [rows][N], where
// row r belongs to RNS limb t = r % l (l limbs per polynomial).
#include "modarith.cuh"

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

__global__ void add_kernel(const uint64_t* a, const uint64_t* b, uint64_t* out, size_t total,
                           int log_n, DivU32 l, const Mod* mods, bool sub) {
  GRID_LOOP(i, total) {
    const int t = (int)umod((uint32_t)(i >> log_n), l);
    const uint64_t q = mods[t].q;
    out[i] = sub ? sub_mod(a[i], b[i], q) : add_mod(a[i], b[i], q);
  }
}

__global__ void mul_pt_kernel(const uint64_t* a, const uint64_t* pt, uint64_t* out, size_t total,
                              int log_n, DivU32 l, const Mod* mods) {
  const size_t N = (size_t)1 << log_n;
  GRID_LOOP(i, total) {
    const int t = (int)umod((uint32_t)(i >> log_n), l);
    out[i] = mul_mod(a[i], pt[(size_t)t * N + (i & (N - 1))], mods[t]);
  }
}

// acc += a * pt (the baby-step accumulation of a diagonal matvec, one pass)
__global__ void mul_pt_acc_kernel(const uint64_t* a, const uint64_t* pt, uint64_t* acc,
                                  size_t total, int log_n, DivU32 l, const Mod* mods) {
  const size_t N = (size_t)1 << log_n;
  GRID_LOOP(i, total) {
    const int t = (int)umod((uint32_t)(i >> log_n), l);
    const uint64_t q = mods[t].q;
    acc[i] = add_mod(acc[i], mul_mod(a[i], pt[(size_t)t * N + (i & (N - 1))], mods[t]), q);
  }
}

// QP_l rows (double-hoisted BSGS): row t of every polynomial uses modulus
// pat[t]; acc = (first ? 0 : acc) + a * pt
__global__ void qp_mul_pt_acc_kernel(const uint64_t* a, const uint64_t* pt, uint64_t* acc,
                                     size_t total, int log_n, DivU32 rows, const int16_t* pat,
                                     const Mod* mods, bool first) {
  const size_t N = (size_t)1 << log_n;
  GRID_LOOP(i, total) {
    const int t = (int)umod((uint32_t)(i >> log_n), rows);
    const Mod& m = mods[pat[t]];
    const uint64_t v = mul_mod(a[i], pt[(size_t)t * N + (i & (N - 1))], m);
    acc[i] = first ? v : add_mod(acc[i], v, m.q);
  }
}

// acc = (first ? 0 : acc) + sum_j a_j * pt_j (one pass over K diagonal
// products; row t of every polynomial uses modulus pat[t])
constexpr int PT_TERMS = 16;
struct PtPairs {
  const uint64_t* a[PT_TERMS];
  const uint64_t* pt[PT_TERMS];
};
__global__ void mul_pt_sum_kernel(PtPairs P, int K, uint64_t* acc, size_t total, int log_n,
                                  DivU32 rows, const int16_t* pat, const Mod* mods, bool first) {
  const size_t N = (size_t)1 << log_n;
  GRID_LOOP(i, total) {
    const int t = (int)umod((uint32_t)(i >> log_n), rows);
    const Mod& m = mods[pat[t]];
    const size_t off = (size_t)t * N + (i & (N - 1));
    uint64_t v = first ? 0 : acc[i];
    for (int j = 0; j < K; j++) v = add_mod(v, mul_mod(P.a[j][i], P.pt[j][off], m), m.q);
    acc[i] = v;
  }
}

// A rotation kept in QP_l: on the Q rows t < l of polynomial 0,
// R += P sigma(c0) (sigma by the NTT-domain permutation perm); the key
// product already in R. identity (perm null): R_k = P c_k on the Q rows and
// 0 on the special primes, for both polynomials.
__global__ void qp_lift_kernel(const uint64_t* ct, uint64_t* R, const uint32_t* perm, size_t B,
                               int log_n, int l, int rows, const uint64_t* pq,
                               const uint64_t* pqs, const Mod* mods) {
  const size_t N = (size_t)1 << log_n;
  const int polys = perm ? 1 : 2;
  GRID_LOOP(i, B * polys * rows * N) {
    const size_t n = i & (N - 1);
    const size_t row = i >> log_n;
    const int t = (int)(row % rows);
    const size_t bk = row / rows;
    const size_t b = bk / polys, k = bk % polys;
    uint64_t* o = R + ((b * 2 + k) * rows + t) * N + n;
    if (t >= l) {
      if (!perm) *o = 0;
      continue;
    }
    const uint64_t q = mods[t].q;
    const uint64_t* src = ct + ((b * 2 + k) * l + t) * N;
    const uint64_t v = mul_shoup(src[perm ? perm[n] : n], pq[t], pqs[t], q);
    *o = perm ? add_mod(*o, v, q) : v;
  }
}

constexpr int LC_TERMS = 16;
struct LincombRes {
  uint64_t v[LC_TERMS][MAX_LIMBS];
};

__global__ void mul_int_kernel(const uint64_t* a, LimbRes k, uint64_t* out, size_t total,
                               int log_n, DivU32 l, const Mod* mods) {
  GRID_LOOP(i, total) {
    const int t = (int)umod((uint32_t)(i >> log_n), l);
    out[i] = mul_shoup(a[i], k.v[t], k.s[t], mods[t].q);
  }
}

// poly 0 of each batch element += k (a constant polynomial is constant in NTT form)
__global__ void add_int_c0_kernel(uint64_t* a, LimbRes k, size_t B, int log_n, DivU32 l,
                                  const Mod* mods) {
  const size_t N = (size_t)1 << log_n;
  const size_t per = (size_t)l.d * N;
  GRID_LOOP(i, B * per) {
    const uint32_t row = (uint32_t)(i >> log_n);
    const size_t b = udiv(row, l);
    const int t = (int)(row - (uint32_t)b * l.d);
    const size_t r = ((size_t)t << log_n) | (i & (N - 1));
    uint64_t* p = a + b * 2 * per + r;
    *p = add_mod(*p, k.v[t], mods[t].q);
  }
}

__global__ void add_pt_c0_kernel(const uint64_t* a, const uint64_t* pt, uint64_t* out, size_t B,
                                 int log_n, DivU32 l2, const Mod* mods) {
  const size_t N = (size_t)1 << log_n;
  const uint32_t l = l2.d / 2;
  GRID_LOOP(i, B * l2.d * N) {
    const uint32_t t = umod((uint32_t)(i >> log_n), l2);  // row within (poly 0, poly 1)
    if (t < l)
      out[i] = add_mod(a[i], pt[((size_t)t << log_n) | (i & (N - 1))], mods[t].q);
    else
      out[i] = a[i];
  }
}

// (a0, a1) x (b0, b1) -> (a0 b0, a0 b1 + a1 b0, a1 b1)
__global__ void tensor_kernel(const uint64_t* a, const uint64_t* b, uint64_t* out, size_t B,
                              int log_n, DivU32 l, const Mod* mods, bool acc) {
  const size_t N = (size_t)1 << log_n;
  const size_t per = (size_t)l.d * N;
  GRID_LOOP(i, B * per) {
    const uint32_t row = (uint32_t)(i >> log_n);
    const size_t bb = udiv(row, l);
    const int t = (int)(row - (uint32_t)bb * l.d);
    const size_t r = ((size_t)t << log_n) | (i & (N - 1));
    const Mod m = mods[t];
    const uint64_t* pa = a + bb * 2 * per + r;
    const uint64_t* pb = b + bb * 2 * per + r;
    const uint64_t a0 = pa[0], a1 = pa[per], b0 = pb[0], b1 = pb[per];
    uint64_t d0 = mul_mod(a0, b0, m);
    uint64_t d1 = add_mod(mul_mod(a0, b1, m), mul_mod(a1, b0, m), m.q);
    uint64_t d2 = mul_mod(a1, b1, m);
    uint64_t* po = out + bb * 3 * per + r;
    if (acc) {
      d0 = add_mod(d0, po[0], m.q);
      d1 = add_mod(d1, po[per], m.q);
      d2 = add_mod(d2, po[2 * per], m.q);
    }
    po[0] = d0;
    po[per] = d1;
    po[2 * per] = d2;
  }
}

struct Ptrs {
  const uint64_t* p[LC_TERMS];
};

__global__ void lincomb_kernel(Ptrs in, LincombRes k, int K, uint64_t* out, size_t total,
                               int log_n, DivU32 l, const Mod* mods) {
  GRID_LOOP(i, total) {
    const int t = (int)umod((uint32_t)(i >> log_n), l);
    const Mod m = mods[t];
    uint64_t acc = 0;
    for (int j = 0; j < K; j++) acc = add_mod(acc, mul_mod(in.p[j][i], k.v[j][t], m), m.q);
    out[i] = acc;
  }
}

__global__ void automorphism_kernel(const uint64_t* in, uint64_t* out, size_t total, int log_n,
                                    const uint32_t* perm) {
  const size_t N = (size_t)1 << log_n;
  GRID_LOOP(i, total) {
    const size_t row = i >> log_n;
    out[i] = in[row * N + perm[i & (N - 1)]];
  }
}

// out = (sigma(a0) + ks0, ks1) per batch element
__global__ void rotate_finish_kernel(const uint64_t* a, const uint64_t* ks, const uint32_t* perm,
                                     uint64_t* out, size_t B, int log_n, DivU32 l, const Mod* mods) {
  const size_t N = (size_t)1 << log_n;
  const size_t per = (size_t)l.d * N;
  GRID_LOOP(i, B * per) {
    const uint32_t row = (uint32_t)(i >> log_n);
    const size_t b = udiv(row, l);
    const int t = (int)(row - (uint32_t)b * l.d);
    const size_t r = ((size_t)t << log_n) | (i & (N - 1));
    const size_t row0 = b * 2 * per + (r & ~(N - 1));
    const uint64_t src = a[row0 + perm[r & (N - 1)]];
    out[b * 2 * per + r] = add_mod(src, ks[b * 2 * per + r], mods[t].q);
    out[b * 2 * per + per + r] = ks[b * 2 * per + per + r];
  }
}

// out = a * pts[(batch index) % K] (pts: up to 16 plaintexts [l][N])
struct PtSet {
  const uint64_t* p[16];
};
__global__ void mul_pt_grouped_kernel(const uint64_t* a, PtSet pts, int K, uint64_t* out,
                                      size_t total, int log_n, DivU32 l, DivU32 l2,
                                      const Mod* mods) {
  const size_t N = (size_t)1 << log_n;
  GRID_LOOP(i, total) {
    const uint32_t row = (uint32_t)(i >> log_n);
    const int t = (int)umod(row, l);
    const int ch = (int)(udiv(row, l2) % (uint32_t)K);
    out[i] = mul_mod(a[i], pts.p[ch][(size_t)t * N + (i & (N - 1))], mods[t]);
  }
}

// acc += a * pts[b % K] per batch element b (chunked first layers)
__global__ void mul_pt_acc_grouped_kernel(const uint64_t* a, PtSet pts, int K, uint64_t* acc,
                                          size_t total, int log_n, DivU32 l, DivU32 l2,
                                          const Mod* mods) {
  const size_t N = (size_t)1 << log_n;
  GRID_LOOP(i, total) {
    const uint32_t row = (uint32_t)(i >> log_n);
    const int t = (int)umod(row, l);
    const int ch = (int)(udiv(row, l2) % (uint32_t)K);
    acc[i] = add_mod(acc[i], mul_mod(a[i], pts.p[ch][(size_t)t * N + (i & (N - 1))], mods[t]),
                     mods[t].q);
  }
}

// out[b] = sum_{c < K} in[b K + c]  (per ciphertext of `per` words)
__global__ void chunk_sum_kernel(const uint64_t* in, uint64_t* out, size_t B, int K, int log_n,
                                 DivU32 l2, const Mod* mods) {
  const size_t N = (size_t)1 << log_n;
  const size_t per = (size_t)l2.d << log_n;
  const uint32_t l = l2.d / 2;
  GRID_LOOP(i, B * per) {
    const uint32_t row = (uint32_t)(i >> log_n);
    const size_t b = udiv(row, l2);
    const uint32_t rr = row - (uint32_t)b * l2.d;  // row within (poly 0, poly 1)
    const int t = (int)(rr < l ? rr : rr - l);
    const size_t r = ((size_t)rr << log_n) | (i & (N - 1));
    const uint64_t q = mods[t].q;
    uint64_t s = in[(b * K) * per + r];
    for (int c = 1; c < K; c++) s = add_mod(s, in[(b * K + c) * per + r], q);
    out[i] = s;
  }
}

// R[p][t][n] = centred(last[p][n]) mod q_t, t < level (last limb mod q_level)
__global__ void rescale_spread_kernel(const uint64_t* last, uint64_t* out, size_t polys,
                                      int log_n, int level, const Mod* mods) {
  const size_t N = (size_t)1 << log_n;
  const uint64_t ql = mods[level].q;
  GRID_LOOP(i, polys * level * N) {
    const size_t p = i / ((size_t)level * N);
    const size_t r = i % ((size_t)level * N);
    const int t = (int)(r >> log_n);
    const uint64_t x = last[p * N + (r & (N - 1))];
    const int64_t v = x > ql / 2 ? -(int64_t)(ql - x) : (int64_t)x;
    out[i] = smod64(v, mods[t].q);
  }
}

// out[p][t] = (in[p][t] - R[p][t]) * q_level^-1 mod q_t
__global__ void rescale_finish_kernel(const uint64_t* in, const uint64_t* R, uint64_t* out,
                                      size_t polys, int log_n, int level, const Mod* mods,
                                      const uint64_t* inv, const uint64_t* invs) {
  const size_t N = (size_t)1 << log_n;
  GRID_LOOP(i, polys * level * N) {
    const size_t p = i / ((size_t)level * N);
    const size_t r = i % ((size_t)level * N);
    const int t = (int)(r >> log_n);
    const uint64_t q = mods[t].q;
    const uint64_t x = in[p * (size_t)(level + 1) * N + r];
    out[i] = mul_shoup(sub_mod(x, R[i], q), inv[t], invs[t], q);
  }
}

__global__ void int_to_rns_kernel(const int64_t* v, uint64_t* out, size_t polys, int rows,
                                  int log_n, const int16_t* pattern, const Mod* mods) {
  const size_t N = (size_t)1 << log_n;
  GRID_LOOP(i, polys * rows * N) {
    const size_t p = i / ((size_t)rows * N);
    const size_t r = (i / N) % rows;
    const int mi = pattern[r];
    out[i] = smod64(v[p * N + (i & (N - 1))], mods[mi].q);
  }
}

LimbRes limb_res(const Ctx& c, int64_t k, int l) {
  if (l > MAX_LIMBS) throw Error(CKKS_ERR_UNSUPPORTED, "more than 64 limbs");
  LimbRes r{};
  for (int t = 0; t < l; t++) {
    const uint64_t q = c.mod[t];
    if (k >= 0) {
      r.v[t] = (uint64_t)k % q;
    } else {
      const uint64_t m = ((uint64_t)(-(k + 1)) + 1) % q;
      r.v[t] = m ? q - m : 0;
    }
    r.s[t] = shoup_h(r.v[t], q);
  }
  return r;
}

}  // namespace

void k_add(Ctx& c, const uint64_t* a, const uint64_t* b, uint64_t* out, size_t rows, int l,
           bool sub) {
  const size_t total = rows * c.N;
  Launch L_(c, K_ADD, 3.0 * total * 8);
  add_kernel<<<grid_for(total), TPB, 0, c.stream>>>(a, b, out, total, c.log_n, divu(l), c.dmod(),
                                                    sub);
  CK_CUDA(cudaGetLastError());
}

void k_mul_pt(Ctx& c, const uint64_t* a, const uint64_t* pt, uint64_t* out, size_t rows, int l) {
  const size_t total = rows * c.N;
  Launch L_(c, K_MUL_PT, 2.0 * total * 8);
  mul_pt_kernel<<<grid_for(total), TPB, 0, c.stream>>>(a, pt, out, total, c.log_n, divu(l),
                                                       c.dmod());
  CK_CUDA(cudaGetLastError());
}

void k_mul_pt_acc(Ctx& c, const uint64_t* a, const uint64_t* pt, uint64_t* acc, size_t rows,
                  int l) {
  const size_t total = rows * c.N;
  Launch L_(c, K_MUL_PT, 3.0 * total * 8, (double)total);
  mul_pt_acc_kernel<<<grid_for(total), TPB, 0, c.stream>>>(a, pt, acc, total, c.log_n, divu(l),
                                                           c.dmod());
  CK_CUDA(cudaGetLastError());
}

void k_qp_mul_pt_acc(Ctx& c, const uint64_t* a, const uint64_t* pt, uint64_t* acc, size_t polys,
                     int level, bool first) {
  ConvTables& T = c.tables(level);
  const size_t total = polys * T.rows * c.N;
  Launch L_(c, K_MUL_PT, (first ? 2.0 : 3.0) * total * 8, (double)total);
  qp_mul_pt_acc_kernel<<<grid_for(total), TPB, 0, c.stream>>>(
      a, pt, acc, total, c.log_n, divu(T.rows), static_cast<const int16_t*>(T.qp_pattern.p),
      c.dmod(), first);
  CK_CUDA(cudaGetLastError());
}

void k_mul_pt_sum(Ctx& c, const std::vector<const uint64_t*>& a,
                  const std::vector<const uint64_t*>& pt, uint64_t* acc, size_t polys, int rows,
                  const int16_t* pattern, bool first) {
  if (a.size() != pt.size() || a.empty()) throw Error(CKKS_ERR_INVALID_ARG, "diagonal products");
  const size_t total = polys * rows * c.N;
  for (size_t s = 0; s < a.size(); s += PT_TERMS) {
    const int K = (int)std::min(a.size() - s, (size_t)PT_TERMS);
    PtPairs P{};
    for (int j = 0; j < K; j++) {
      P.a[j] = a[s + j];
      P.pt[j] = pt[s + j];
    }
    const bool f = first && s == 0;
    Launch L_(c, K_MUL_PT, (K + (f ? 1.0 : 2.0)) * total * 8 + K * (double)rows * c.N * 8,
              (double)K * total);
    mul_pt_sum_kernel<<<grid_for(total), TPB, 0, c.stream>>>(P, K, acc, total, c.log_n, divu(rows),
                                                             pattern, c.dmod(), f);
    CK_CUDA(cudaGetLastError());
  }
}

void k_qp_lift(Ctx& c, const uint64_t* ct, size_t B, int level, const uint32_t* perm, uint64_t* R) {
  ConvTables& T = c.tables(level);
  const int l = T.l;
  const size_t total = B * (perm ? 1 : 2) * T.rows * c.N;
  Launch L_(c, K_ROT_FINISH, (perm ? 3.0 : 2.0) * total * 8);
  qp_lift_kernel<<<grid_for(total), TPB, 0, c.stream>>>(ct, R, perm, B, c.log_n, l, T.rows,
                                                        T.md_pq.u64(), T.md_pq_s.u64(), c.dmod());
  CK_CUDA(cudaGetLastError());
}

void k_mul_int(Ctx& c, const uint64_t* a, int64_t k, uint64_t* out, size_t rows, int l) {
  const size_t total = rows * c.N;
  Launch L_(c, K_MUL_INT, 2.0 * total * 8);
  mul_int_kernel<<<grid_for(total), TPB, 0, c.stream>>>(a, limb_res(c, k, l), out, total, c.log_n,
                                                        divu(l), c.dmod());
  CK_CUDA(cudaGetLastError());
}

void k_mul_limbs(Ctx& c, const uint64_t* a, const std::vector<uint64_t>& res, uint64_t* out,
                 size_t rows, int l) {
  if (l > MAX_LIMBS || (int)res.size() < l) throw Error(CKKS_ERR_UNSUPPORTED, "limb constants");
  LimbRes r{};
  for (int t = 0; t < l; t++) {
    r.v[t] = res[t];
    r.s[t] = shoup_h(res[t], c.mod[t]);
  }
  const size_t total = rows * c.N;
  Launch L_(c, K_MUL_INT, 2.0 * total * 8);
  mul_int_kernel<<<grid_for(total), TPB, 0, c.stream>>>(a, r, out, total, c.log_n, divu(l),
                                                        c.dmod());
  CK_CUDA(cudaGetLastError());
}

void k_add_int_c0(Ctx& c, uint64_t* a, int64_t k, size_t B, int l) {
  Launch L_(c, K_ADD, 2.0 * B * l * c.N * 8);
  add_int_c0_kernel<<<grid_for(B * l * c.N), TPB, 0, c.stream>>>(a, limb_res(c, k, l), B, c.log_n,
                                                                 divu(l), c.dmod());
  CK_CUDA(cudaGetLastError());
}

void k_add_pt_c0(Ctx& c, const uint64_t* a, const uint64_t* pt, uint64_t* out, size_t B, int l) {
  Launch L_(c, K_ADD, 5.0 * B * l * c.N * 8);
  add_pt_c0_kernel<<<grid_for(B * 2 * l * c.N), TPB, 0, c.stream>>>(a, pt, out, B, c.log_n,
                                                                     divu(2 * l), c.dmod());
  CK_CUDA(cudaGetLastError());
}

void k_tensor(Ctx& c, const uint64_t* a, const uint64_t* b, uint64_t* out, size_t B, int l,
              bool accumulate) {
  Launch L_(c, K_TENSOR, (accumulate ? 10.0 : 7.0) * B * l * c.N * 8);
  tensor_kernel<<<grid_for(B * l * c.N), TPB, 0, c.stream>>>(a, b, out, B, c.log_n, divu(l),
                                                             c.dmod(), accumulate);
  CK_CUDA(cudaGetLastError());
}

void k_lincomb_int(Ctx& c, const std::vector<const uint64_t*>& in, const std::vector<int64_t>& k,
                   uint64_t* out, size_t rows, int l) {
  if (in.size() > (size_t)LC_TERMS || in.size() != k.size() || in.empty())
    throw Error(CKKS_ERR_INVALID_ARG, "lincomb: 1..16 terms");
  if (l > MAX_LIMBS) throw Error(CKKS_ERR_UNSUPPORTED, "more than 64 limbs");
  Ptrs P{};
  LincombRes C;  // by-value kernel argument (8 KiB)
  for (size_t j = 0; j < in.size(); j++) {
    P.p[j] = in[j];
    const LimbRes r = limb_res(c, k[j], l);
    for (int t = 0; t < l; t++) C.v[j][t] = r.v[t];
  }
  const size_t total = rows * c.N;
  Launch L_(c, K_LINCOMB, (in.size() + 1.0) * total * 8);
  lincomb_kernel<<<grid_for(total), TPB, 0, c.stream>>>(P, C, (int)in.size(), out, total, c.log_n,
                                                        divu(l), c.dmod());
  CK_CUDA(cudaGetLastError());
}

void k_copy_limbs(Ctx& c, const uint64_t* in, int l_in, uint64_t* out, int l_out, size_t polys) {
  const size_t w = (size_t)l_out * c.N * 8;
  Launch L_(c, K_COPY, 2.0 * w * polys);
  CK_CUDA(cudaMemcpy2DAsync(out, w, in, (size_t)l_in * c.N * 8, w, polys, cudaMemcpyDeviceToDevice,
                            c.stream));
}

void k_automorphism(Ctx& c, const uint64_t* in, uint64_t* out, size_t rows, const uint32_t* perm) {
  const size_t total = rows * c.N;
  Launch L_(c, K_AUTO, 2.0 * total * 8);
  automorphism_kernel<<<grid_for(total), TPB, 0, c.stream>>>(in, out, total, c.log_n, perm);
  CK_CUDA(cudaGetLastError());
}

void k_mul_pt_grouped(Ctx& c, const uint64_t* a, const std::vector<const uint64_t*>& pts,
                      uint64_t* out, size_t B, int l) {
  if (pts.empty() || pts.size() > 16) throw Error(CKKS_ERR_UNSUPPORTED, "1..16 plaintexts");
  PtSet P{};
  for (size_t k = 0; k < pts.size(); k++) P.p[k] = pts[k];
  const size_t total = B * 2 * (size_t)l * c.N;
  Launch L_(c, K_MUL_PT, 2.0 * total * 8, (double)total);
  mul_pt_grouped_kernel<<<grid_for(total), TPB, 0, c.stream>>>(a, P, (int)pts.size(), out, total,
                                                                c.log_n, divu(l), divu(2 * l),
                                                                c.dmod());
  CK_CUDA(cudaGetLastError());
}

void k_mul_pt_acc_grouped(Ctx& c, const uint64_t* a, const std::vector<const uint64_t*>& pts,
                          uint64_t* acc, size_t B, int l) {
  if (pts.empty() || pts.size() > 16) throw Error(CKKS_ERR_UNSUPPORTED, "1..16 plaintexts");
  PtSet P{};
  for (size_t k = 0; k < pts.size(); k++) P.p[k] = pts[k];
  const size_t total = B * 2 * (size_t)l * c.N;
  Launch L_(c, K_MUL_PT, 3.0 * total * 8, (double)total);
  mul_pt_acc_grouped_kernel<<<grid_for(total), TPB, 0, c.stream>>>(a, P, (int)pts.size(), acc,
                                                                    total, c.log_n, divu(l),
                                                                    divu(2 * l), c.dmod());
  CK_CUDA(cudaGetLastError());
}

void k_chunk_sum(Ctx& c, const uint64_t* in, uint64_t* out, size_t B, int K, int l) {
  const size_t total = B * 2 * (size_t)l * c.N;
  Launch L_(c, K_ADD, (K + 1.0) * total * 8);
  chunk_sum_kernel<<<grid_for(total), TPB, 0, c.stream>>>(in, out, B, K, c.log_n, divu(2 * l),
                                                          c.dmod());
  CK_CUDA(cudaGetLastError());
}

void k_rotate_finish(Ctx& c, const uint64_t* a, const uint64_t* ks, const uint32_t* perm,
                     uint64_t* out, size_t B, int l) {
  Launch L_(c, K_ROT_FINISH, 5.0 * B * l * c.N * 8);
  rotate_finish_kernel<<<grid_for(B * l * c.N), TPB, 0, c.stream>>>(a, ks, perm, out, B, c.log_n,
                                                                    divu(l), c.dmod());
  CK_CUDA(cudaGetLastError());
}

void k_rescale_spread(Ctx& c, const uint64_t* last, uint64_t* out, size_t polys, int level) {
  Launch L_(c, K_RS_SPREAD, (1.0 + level) * polys * c.N * 8);
  rescale_spread_kernel<<<grid_for(polys * level * c.N), TPB, 0, c.stream>>>(last, out, polys,
                                                                            c.log_n, level, c.dmod());
  CK_CUDA(cudaGetLastError());
}

void k_rescale_finish(Ctx& c, const uint64_t* in, const uint64_t* r, uint64_t* out, size_t polys,
                      int level, const uint64_t* inv, const uint64_t* invs) {
  Launch L_(c, K_RS_FINISH, 3.0 * level * polys * c.N * 8);
  rescale_finish_kernel<<<grid_for(polys * level * c.N), TPB, 0, c.stream>>>(
      in, r, out, polys, c.log_n, level, c.dmod(), inv, invs);
  CK_CUDA(cudaGetLastError());
}

void k_int_to_rns(Ctx& c, const int64_t* v, uint64_t* out, size_t polys, int rows,
                  const int16_t* pattern) {
  Launch L_(c, K_INT_RNS, (1.0 + rows) * polys * c.N * 8);
  int_to_rns_kernel<<<grid_for(polys * rows * c.N), TPB, 0, c.stream>>>(v, out, polys, rows,
                                                                       c.log_n, pattern, c.dmod());
  CK_CUDA(cudaGetLastError());
}

}  // namespace ck
