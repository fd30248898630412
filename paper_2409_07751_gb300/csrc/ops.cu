// Ciphertext operations with level and scale bookkeeping (see ops.h).
#include <math.h>

#include <algorithm>

#include "ops.h"

namespace ck {

Ct ct_alloc(Ctx& c, size_t B, int level, double scale) {
  if (level < 0 || level > c.L) throw Error(CKKS_ERR_LEVEL, "level out of range");
  Ct r(new ckks_ct{&c, DevBuf(), B, level, scale});
  r->d = DevBuf(&c, r->words() * 8);
  return r;
}

Ct ct_copy(Ctx& c, const ckks_ct& a) {
  Ct r = ct_alloc(c, a.B, a.level, a.scale);
  CK_CUDA(cudaMemcpyAsync(r->d.p, a.d.p, r->d.bytes, cudaMemcpyDeviceToDevice, c.stream));
  return r;
}

void check_pair(const ckks_ct& a, const ckks_ct& b) {
  if (a.B != b.B) throw Error(CKKS_ERR_INVALID_ARG, "batch sizes differ");
  if (a.level != b.level) throw Error(CKKS_ERR_LEVEL, "levels differ");
  if (fabs(a.scale / b.scale - 1.0) > SNAP) throw Error(CKKS_ERR_SCALE, "scales differ");
}

int64_t round_const(double v, double scale) {
  const double r = rint(v * scale);
  if (!(fabs(r) < 9.2e18)) throw Error(CKKS_ERR_OVERFLOW, "constant does not fit its scale");
  return (int64_t)r;
}

double plain_scale(const Ctx& c, double ct_scale, int level) {
  if (level < 1 || level > c.L) throw Error(CKKS_ERR_LEVEL, "level exhausted");
  return (c.delta[level - 1] * (double)c.mod[level]) / ct_scale;
}

DevBuf encode_vec(Ctx& c, const double* host, size_t n, int level, double scale) {
  DevBuf pt(&c, (size_t)(level + 1) * c.N * 8);
  DevBuf v(&c, std::max<size_t>(n, 1) * 8);
  if (n) CK_CUDA(cudaMemcpyAsync(v.p, host, n * 8, cudaMemcpyHostToDevice, c.stream));
  const int rc = encode(c, static_cast<const double*>(v.p), 1, n, level, scale, pt.u64());
  if (rc != CKKS_OK) throw Error(rc, "plaintext does not fit its scale");
  return pt;
}

DevBuf encode_vec_qp(Ctx& c, const double* host, size_t n, int level, double scale) {
  ConvTables& T = c.tables(level);
  DevBuf pt(&c, (size_t)T.rows * c.N * 8);
  DevBuf v(&c, std::max<size_t>(n, 1) * 8);
  if (n) CK_CUDA(cudaMemcpyAsync(v.p, host, n * 8, cudaMemcpyHostToDevice, c.stream));
  const int rc = encode_rows(c, static_cast<const double*>(v.p), 1, n, T.rows,
                             static_cast<const int16_t*>(T.qp_pattern.p), scale, pt.u64());
  if (rc != CKKS_OK) throw Error(rc, "plaintext does not fit its scale");
  return pt;
}

Ct op_add(Ctx& c, const ckks_ct& a, const ckks_ct& b, bool sub) {
  check_pair(a, b);
  Ct r = ct_alloc(c, a.B, a.level, a.scale);
  k_add(c, a.d.u64(), b.d.u64(), r->d.u64(), a.B * 2 * (a.level + 1), a.level + 1, sub);
  return r;
}

Ct op_mul_int(Ctx& c, const ckks_ct& a, int64_t k) {
  Ct r = ct_alloc(c, a.B, a.level, a.scale);
  k_mul_int(c, a.d.u64(), k, r->d.u64(), a.B * 2 * (a.level + 1), a.level + 1);
  return r;
}

Ct op_add_const(Ctx& c, const ckks_ct& a, double v) {
  Ct r = ct_copy(c, a);
  k_add_int_c0(c, r->d.u64(), round_const(v, a.scale), a.B, a.level + 1);
  return r;
}

Ct op_add_pt(Ctx& c, const ckks_ct& a, const uint64_t* pt) {
  Ct r = ct_alloc(c, a.B, a.level, a.scale);
  k_add_pt_c0(c, a.d.u64(), pt, r->d.u64(), a.B, a.level + 1);
  return r;
}

Ct op_mod_drop(Ctx& c, const ckks_ct& a, int level) {
  if (level > a.level) throw Error(CKKS_ERR_LEVEL, "mod_drop cannot raise the level");
  Ct r = ct_alloc(c, a.B, level, a.scale);
  k_copy_limbs(c, a.d.u64(), a.level + 1, r->d.u64(), level + 1, a.B * 2);
  return r;
}

Ct op_rescale(Ctx& c, const ckks_ct& a) {
  const int lv = a.level;
  if (lv < 1) throw Error(CKKS_ERR_LEVEL, "level exhausted");
  const size_t polys = a.B * 2;
  DevBuf last(&c, polys * c.N * 8);
  CK_CUDA(cudaMemcpy2DAsync(last.p, c.N * 8, a.d.u64() + (size_t)lv * c.N,
                            (size_t)(lv + 1) * c.N * 8, c.N * 8, polys, cudaMemcpyDeviceToDevice,
                            c.stream));
  ntt_inverse(c, last.u64(), polys, c.iota() + lv, 1);
  double s = a.scale / (double)c.mod[lv];
  const double d = c.delta[lv - 1];
  if (fabs(s / d - 1.0) < SNAP) s = d;
  if (ntt_fused_available(c)) {
    Ct r = ct_alloc(c, a.B, lv - 1, s);
    ntt_rescale_fused(c, a.d.u64(), last.u64(), polys, lv, r->d.u64());
    return r;
  }
  DevBuf R(&c, polys * lv * c.N * 8);
  k_rescale_spread(c, last.u64(), R.u64(), polys, lv);
  ntt_forward(c, R.u64(), polys * lv, c.iota(), lv);
  Ct r = ct_alloc(c, a.B, lv - 1, s);
  k_rescale_finish(c, a.d.u64(), R.u64(), r->d.u64(), polys, lv,
                   c.d_rs_inv.u64() + (size_t)lv * (c.L + 1),
                   c.d_rs_invs.u64() + (size_t)lv * (c.L + 1));
  return r;
}

Ct op_mul_pt(Ctx& c, const ckks_ct& a, const uint64_t* pt, double pt_scale) {
  Ct t = ct_alloc(c, a.B, a.level, a.scale * pt_scale);
  k_mul_pt(c, a.d.u64(), pt, t->d.u64(), a.B * 2 * (a.level + 1), a.level + 1);
  return op_rescale(c, *t);
}

// rescale by q_r of k a restricted to limbs 0..r (r <= a.level), the product
// carrying `scale`: the limb drop and the integer factor are folded into the
// rescale's transforms (same residues as mod-drop, multiply, rescale)
static Ct scale_rescale(Ctx& c, const ckks_ct& a, int r, int64_t k, double scale) {
  if (r < 1 || r > a.level) throw Error(CKKS_ERR_LEVEL, "level exhausted");
  if (!ntt_fused_available(c)) {
    Ct b = r < a.level ? op_mod_drop(c, a, r) : nullptr;
    Ct t = op_mul_int(c, b ? *b : a, k);
    t->scale = scale;
    return op_rescale(c, *t);
  }
  double s = scale / (double)c.mod[r];
  const double d = c.delta[r - 1];
  if (fabs(s / d - 1.0) < SNAP) s = d;
  const size_t polys = a.B * 2;
  const size_t stride = (size_t)(a.level + 1) * c.N;
  const uint64_t* kc = c.scaled_consts(r, k);
  DevBuf last(&c, polys * c.N * 8);
  ntt_inverse_post(c, last.u64(), polys, c.iota() + r, 1, kc, kc + 1, SIZE_MAX,
                   a.d.u64() + (size_t)r * c.N, stride);
  Ct out = ct_alloc(c, a.B, r - 1, s);
  ntt_rescale_scaled_fused(c, a.d.u64(), stride, last.u64(), polys, r, kc + 2, kc + 2 + r,
                           out->d.u64());
  return out;
}

Ct op_mul_const(Ctx& c, const ckks_ct& a, double v) {
  const double S = plain_scale(c, a.scale, a.level);
  return scale_rescale(c, a, a.level, round_const(v, S), a.scale * S);
}

Ct op_level_down(Ctx& c, const ckks_ct& a, int level) {
  if (level == a.level && fabs(a.scale / c.delta[level] - 1.0) < SNAP) return ct_copy(c, a);
  if (level >= a.level) throw Error(CKKS_ERR_LEVEL, "level_down needs a lower level");
  const double S = plain_scale(c, a.scale, level + 1);
  return scale_rescale(c, a, level + 1, round_const(1.0, S), a.scale * S);
}

Ct op_lincomb(Ctx& c, const std::vector<const ckks_ct*>& in, const std::vector<double>& k,
              double cst, int level) {
  if (in.empty()) throw Error(CKKS_ERR_INVALID_ARG, "lincomb of nothing");
  if (level < 0) {
    level = in[0]->level;
    for (auto* p : in) level = std::min(level, p->level);
    level -= 1;
  }
  if (level < 0) throw Error(CKKS_ERR_LEVEL, "level exhausted");
  const int top = level + 1;
  const size_t B = in[0]->B;
  std::vector<Ct> dropped;
  std::vector<const uint64_t*> ptrs;
  std::vector<int64_t> ks;
  for (size_t i = 0; i < in.size(); i++) {
    if (k[i] == 0.0) continue;
    const ckks_ct* p = in[i];
    if (p->B != B) throw Error(CKKS_ERR_INVALID_ARG, "batch sizes differ");
    if (p->level < top) throw Error(CKKS_ERR_LEVEL, "lincomb input below target");
    const double S = (c.delta[level] * (double)c.mod[top]) / p->scale;
    ks.push_back(round_const(k[i], S));
    if (p->level > top) {
      dropped.push_back(op_mod_drop(c, *p, top));
      ptrs.push_back(dropped.back()->d.u64());
    } else {
      ptrs.push_back(p->d.u64());
    }
  }
  Ct acc = ct_alloc(c, B, top, c.delta[level] * (double)c.mod[top]);
  const size_t rows = B * 2 * (top + 1);
  if (ptrs.empty()) {
    CK_CUDA(cudaMemsetAsync(acc->d.p, 0, acc->d.bytes, c.stream));
  } else {
    // at most 16 terms per pass
    for (size_t s = 0; s < ptrs.size(); s += 16) {
      const size_t e = std::min(ptrs.size(), s + 16);
      std::vector<const uint64_t*> pp(ptrs.begin() + s, ptrs.begin() + e);
      std::vector<int64_t> kk(ks.begin() + s, ks.begin() + e);
      if (s == 0) {
        k_lincomb_int(c, pp, kk, acc->d.u64(), rows, top + 1);
      } else {
        Ct part = ct_alloc(c, B, top, acc->scale);
        k_lincomb_int(c, pp, kk, part->d.u64(), rows, top + 1);
        k_add(c, acc->d.u64(), part->d.u64(), acc->d.u64(), rows, top + 1, false);
      }
    }
  }
  Ct out = op_rescale(c, *acc);
  out->scale = c.delta[level];
  if (cst != 0.0) out = op_add_const(c, *out, cst);
  return out;
}

static DevBuf tensor(Ctx& c, const ckks_ct& a, const ckks_ct& b) {
  if (a.level != b.level || a.B != b.B) throw Error(CKKS_ERR_LEVEL, "tensor needs equal levels");
  DevBuf d(&c, a.B * 3 * (a.level + 1) * c.N * 8);
  k_tensor(c, a.d.u64(), b.d.u64(), d.u64(), a.B, a.level + 1, false);
  return d;
}

// d: [B][3][l][N] -> (d0, d1) + KeySwitch(d2)
static Ct relinearise(Ctx& c, const ckks_keys& keys, const DevBuf& d, size_t B, int level,
                      double scale) {
  const int l = level + 1;
  ConvTables& T = c.tables(level);
  DevBuf d2(&c, B * l * c.N * 8);
  CK_CUDA(cudaMemcpy2DAsync(d2.p, (size_t)l * c.N * 8, d.u64() + 2 * (size_t)l * c.N,
                            3 * (size_t)l * c.N * 8, (size_t)l * c.N * 8, B,
                            cudaMemcpyDeviceToDevice, c.stream));
  DevBuf ext(&c, B * T.beta * T.rows * c.N * 8);
  modup(c, d2.u64(), B, level, ext.u64());
  d2.reset();
  Ct ks = ct_alloc(c, B, level, scale);
  DevBuf kt;
  keyswitch_ext(c, ext.u64(), B, level, switch_key_words(c, keys, 0, kt), 0, ks->d.u64());
  ext.reset();
  // (d0, d1) of each batch element sit at the start of its 3-poly block
  Ct r = ct_alloc(c, B, level, scale);
  CK_CUDA(cudaMemcpy2DAsync(r->d.p, 2 * (size_t)l * c.N * 8, d.p, 3 * (size_t)l * c.N * 8,
                            2 * (size_t)l * c.N * 8, B, cudaMemcpyDeviceToDevice, c.stream));
  k_add(c, r->d.u64(), ks->d.u64(), r->d.u64(), B * 2 * l, l, false);
  return r;
}

// d: [B][3][l][N] at `level` -> relinearised and rescaled to level - 1 in one
// division by P q_level (ModUp of d2, key product, merged ModDown + rescale)
static Ct relin_rescale(Ctx& c, const ckks_keys& keys, const DevBuf& d, size_t B, int level,
                        double scale) {
  if (level < 1) throw Error(CKKS_ERR_LEVEL, "level exhausted");
  const int l = level + 1;
  ConvTables& T = c.tables(level);
  DevBuf ext(&c, B * T.beta * T.rows * c.N * 8);
  // d2 of batch element b sits at d + (3b + 2) l N
  modup(c, d.u64() + 2 * (size_t)l * c.N, B, level, ext.u64(), 3 * (size_t)l * c.N);
  double s = scale / (double)c.mod[level];
  const double dl = c.delta[level - 1];
  if (fabs(s / dl - 1.0) < SNAP) s = dl;
  Ct r = ct_alloc(c, B, level - 1, s);
  DevBuf kt;
  relin_rescale_ext(c, d.u64(), ext.u64(), B, level, switch_key_words(c, keys, 0, kt),
                    r->d.u64());
  return r;
}

Ct op_mul_relin(Ctx& c, const ckks_keys& keys, const ckks_ct& a, const ckks_ct& b) {
  DevBuf d = tensor(c, a, b);
  return relinearise(c, keys, d, a.B, a.level, a.scale * b.scale);
}

Ct op_mul(Ctx& c, const ckks_keys& keys, const ckks_ct& a, const ckks_ct& b) {
  const int lv = std::min(a.level, b.level);
  Ct a2 = op_level_down(c, a, lv);
  Ct b2 = op_level_down(c, b, lv);
  DevBuf d = tensor(c, *a2, *b2);
  return relin_rescale(c, keys, d, a2->B, lv, a2->scale * b2->scale);
}

Ct op_mul_sum(Ctx& c, const ckks_keys& keys,
              const std::vector<std::pair<const ckks_ct*, const ckks_ct*>>& pairs) {
  int lv = 1 << 30;
  for (auto& p : pairs) lv = std::min(lv, std::min(p.first->level, p.second->level));
  DevBuf acc;
  double scale = 0;
  size_t B = pairs[0].first->B;
  for (size_t i = 0; i < pairs.size(); i++) {
    Ct a = op_level_down(c, *pairs[i].first, lv);
    Ct b = op_level_down(c, *pairs[i].second, lv);
    if (i == 0) {
      acc = tensor(c, *a, *b);
      scale = a->scale * b->scale;
    } else {
      k_tensor(c, a->d.u64(), b->d.u64(), acc.u64(), B, lv + 1, true);
    }
  }
  return relin_rescale(c, keys, acc, B, lv, scale);
}

std::vector<Ct> op_rotate_many(Ctx& c, const ckks_keys& keys, const ckks_ct& a,
                               const std::vector<int64_t>& steps) {
  std::vector<uint64_t> g;
  for (int64_t t : steps) g.push_back(c.galois(t));
  return op_galois_many(c, keys, a, g);
}

std::vector<Ct> op_galois_many(Ctx& c, const ckks_keys& keys, const ckks_ct& a,
                               const std::vector<uint64_t>& galois) {
  std::vector<Ct> out;
  const int l = a.level + 1;
  ConvTables& T = c.tables(a.level);
  DevBuf ext;
  for (uint64_t g : galois) {
    if (g == 1) {
      out.push_back(ct_copy(c, a));
      continue;
    }
    DevBuf kt;
    const uint64_t* key = switch_key_words(c, keys, g, kt);
    if (!ext.p) {
      ext = DevBuf(&c, a.B * T.beta * T.rows * c.N * 8);
      // c1 of batch element b sits at a + (2b + 1) l N
      modup(c, a.d.u64() + (size_t)l * c.N, a.B, a.level, ext.u64(), 2 * (size_t)l * c.N);
    }
    Ct ks = ct_alloc(c, a.B, a.level, a.scale);
    keyswitch_ext(c, ext.u64(), a.B, a.level, key, g, ks->d.u64());
    Ct r = ct_alloc(c, a.B, a.level, a.scale);
    // c0' = sigma(c0) + ks0, c1' = ks1
    k_rotate_finish(c, a.d.u64(), ks->d.u64(), c.perm(g), r->d.u64(), a.B, l);
    out.push_back(std::move(r));
  }
  return out;
}

Ct op_rotate(Ctx& c, const ckks_keys& keys, const ckks_ct& a, int64_t step) {
  auto v = op_rotate_many(c, keys, a, {step});
  return std::move(v[0]);
}

Ct op_concat(Ctx& c, const std::vector<const ckks_ct*>& in) {
  size_t B = 0;
  for (auto* p : in) {
    if (p->level != in[0]->level) throw Error(CKKS_ERR_LEVEL, "concat needs equal levels");
    B += p->B;
  }
  Ct r = ct_alloc(c, B, in[0]->level, in[0]->scale);
  size_t off = 0;
  for (auto* p : in) {
    CK_CUDA(cudaMemcpyAsync(r->d.u64() + off, p->d.p, p->d.bytes, cudaMemcpyDeviceToDevice, c.stream));
    off += p->words();
  }
  return r;
}

}  // namespace ck
