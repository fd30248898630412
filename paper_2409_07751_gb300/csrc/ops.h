// Ciphertext operations with level and scale bookkeeping.
//
// Scale rule: a ciphertext at level l carries the canonical scale Delta_l
// (Delta_{l-1} = Delta_l^2 / q_l). Plaintext operands of a product are
// encoded at the scale that lands the rescaled product on Delta_{l-1};
// moving to a lower level multiplies by an integer constant and rescales;
// a rescaled scale within 2^-30 of the canonical one is snapped to it.
#pragma once
#include <utility>

#include "internal.h"

namespace ck {

using Ct = std::unique_ptr<ckks_ct>;

constexpr double SNAP = 1.0 / 1073741824.0;  // 2^-30

Ct ct_alloc(Ctx& c, size_t B, int level, double scale);
Ct ct_copy(Ctx& c, const ckks_ct& a);
void check_pair(const ckks_ct& a, const ckks_ct& b);

int64_t round_const(double v, double scale);
double plain_scale(const Ctx& c, double ct_scale, int level);

// plaintext [l][N] (device) of a real vector at `level` and `scale`
DevBuf encode_vec(Ctx& c, const double* host, size_t n, int level, double scale);
// the same over QP_level ([l + alpha][N]: Q limbs, then the special primes)
DevBuf encode_vec_qp(Ctx& c, const double* host, size_t n, int level, double scale);

Ct op_add(Ctx& c, const ckks_ct& a, const ckks_ct& b, bool sub);
Ct op_mul_int(Ctx& c, const ckks_ct& a, int64_t k);
Ct op_add_const(Ctx& c, const ckks_ct& a, double v);
Ct op_add_pt(Ctx& c, const ckks_ct& a, const uint64_t* pt);
Ct op_mod_drop(Ctx& c, const ckks_ct& a, int level);
Ct op_rescale(Ctx& c, const ckks_ct& a);
// a (x) pt then rescale; pt must be encoded at plain_scale(a.scale, a.level)
Ct op_mul_pt(Ctx& c, const ckks_ct& a, const uint64_t* pt, double pt_scale);
Ct op_mul_const(Ctx& c, const ckks_ct& a, double v);
Ct op_level_down(Ctx& c, const ckks_ct& a, int level);
Ct op_lincomb(Ctx& c, const std::vector<const ckks_ct*>& in, const std::vector<double>& k,
              double cst, int level);
Ct op_mul_relin(Ctx& c, const ckks_keys& keys, const ckks_ct& a, const ckks_ct& b);
Ct op_mul(Ctx& c, const ckks_keys& keys, const ckks_ct& a, const ckks_ct& b);
Ct op_mul_sum(Ctx& c, const ckks_keys& keys,
              const std::vector<std::pair<const ckks_ct*, const ckks_ct*>>& pairs);
std::vector<Ct> op_rotate_many(Ctx& c, const ckks_keys& keys, const ckks_ct& a,
                               const std::vector<int64_t>& steps);
Ct op_rotate(Ctx& c, const ckks_keys& keys, const ckks_ct& a, int64_t step);
// the automorphisms X -> X^g (g odd) of a, sharing one ModUp
std::vector<Ct> op_galois_many(Ctx& c, const ckks_keys& keys, const ckks_ct& a,
                               const std::vector<uint64_t>& galois);
Ct op_concat(Ctx& c, const std::vector<const ckks_ct*>& in);

// keys.cu: hamming > 0 draws a sparse secret of that weight; conjugation
// adds the key of the Galois element 2N - 1; a_seed != 0 draws the switching
// keys' uniform halves from that public seed
std::unique_ptr<ckks_keys> keygen(Ctx& c, uint64_t seed, const std::vector<int64_t>& steps,
                                  int hamming = 0, bool conjugation = false, uint64_t a_seed = 0);
// the switching key of Galois element g (0: relinearisation) as
// [beta_max][2][n_qp][N] words: the stored key, or for seed-compressed keys
// the b halves with the a halves regenerated into `tmp`
// (CKKS_ERR_MISSING_KEY if there is none)
const uint64_t* switch_key_words(Ctx& c, const ckks_keys& keys, uint64_t g, DevBuf& tmp);
// drop the uniform halves of every switching key (keys with a public seed)
void keys_compress(Ctx& c, ckks_keys& keys);
Ct encrypt(Ctx& c, const ckks_keys& keys, const double* values, size_t B, size_t n, int level,
           uint64_t seed, uint64_t first_index);
void decrypt(Ctx& c, const ckks_keys& keys, const ckks_ct& ct, double* out, size_t n);

// elementwise.cu (extra entry points)
void k_mul_int(Ctx& c, const uint64_t* a, int64_t k, uint64_t* out, size_t rows, int l);
void k_add_int_c0(Ctx& c, uint64_t* a, int64_t k, size_t B, int l);
// limb t of every row times res[t] (an integer of any size, by its residues)
void k_mul_limbs(Ctx& c, const uint64_t* a, const std::vector<uint64_t>& res, uint64_t* out,
                 size_t rows, int l);
void k_lincomb_int(Ctx& c, const std::vector<const uint64_t*>& in, const std::vector<int64_t>& k,
                   uint64_t* out, size_t rows, int l);
void k_rotate_finish(Ctx& c, const uint64_t* a, const uint64_t* ks, const uint32_t* perm,
                     uint64_t* out, size_t B, int l);
// batch element b of a [B][2][l][N] batch multiplied by pts[b % pts.size()]
// acc += a * pt (one pass), and the per-chunk form of it
void k_mul_pt_acc(Ctx& c, const uint64_t* a, const uint64_t* pt, uint64_t* acc, size_t rows,
                  int l);
void k_mul_pt_acc_grouped(Ctx& c, const uint64_t* a, const std::vector<const uint64_t*>& pts,
                          uint64_t* acc, size_t B, int l);
void k_mul_pt_grouped(Ctx& c, const uint64_t* a, const std::vector<const uint64_t*>& pts,
                      uint64_t* out, size_t B, int l);
// double-hoisted BSGS over QP_level rows ([polys][l + alpha][N]): acc (=) +=
// a * pt; a rotation kept in QP (R holds the key product; perm null: the
// identity, R = P c)
void k_qp_mul_pt_acc(Ctx& c, const uint64_t* a, const uint64_t* pt, uint64_t* acc, size_t polys,
                     int level, bool first);
void k_qp_lift(Ctx& c, const uint64_t* ct, size_t B, int level, const uint32_t* perm, uint64_t* R);
// acc = (first ? 0 : acc) + sum_j a[j] * pt[j] over polys polynomials of
// `rows` rows (row t modulus pattern[t]; pt[j]: [rows][N]), one pass per 16
// products
void k_mul_pt_sum(Ctx& c, const std::vector<const uint64_t*>& a,
                  const std::vector<const uint64_t*>& pt, uint64_t* acc, size_t polys, int rows,
                  const int16_t* pattern, bool first);
// out[b] = sum_c in[b K + c]
void k_chunk_sum(Ctx& c, const uint64_t* in, uint64_t* out, size_t B, int K, int l);
void k_rescale_finish(Ctx& c, const uint64_t* in, const uint64_t* r, uint64_t* out, size_t polys,
                      int level, const uint64_t* inv, const uint64_t* invs);

// kan.cu: sum_j a_j T_j(y) (Paterson-Stockmeyer over the Chebyshev basis)
// and the levels it takes
Ct cheb_eval(Ctx& c, const ckks_keys& keys, const ckks_ct& y, const std::vector<double>& a);
int cheb_levels(int degree);

// boot.cu: the whole refresh of a level-0 batch with a plan, and the
// packed refresh of a batch whose ciphertexts carry n_out leading slots
Ct bootstrap(Ctx& c, const ckks_keys& keys, const ckks_boot& b, const ckks_ct& in);
Ct refresh_packed(Ctx& c, const ckks_keys& keys, const ckks_boot& b, const ckks_ct& in,
                  int n_out);

// capi.cu: translates the exception being handled into an error code and
// records its message for ckks_last_error; call only inside a catch block
int api_error();

}  // namespace ck
