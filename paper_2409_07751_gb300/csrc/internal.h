// Internal types of the GB300 RNS-CKKS library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/ckks_kan.h"

namespace ck {

// Per-modulus constants visible to kernels.
// most key-switching digits a key inner product takes (keys staged in shared memory)
constexpr int MAX_DIGITS = 32;

struct Mod {
  uint64_t q;
  uint64_t mu;   // floor(2^(2s) / q), Barrett
  uint32_t s;    // bit length of q
  uint32_t pad;
  uint64_t t64;  // 2^64 mod q
};

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void cuda_check(cudaError_t e, const char* what);
#define CK_CUDA(x) ::ck::cuda_check((x), #x)

struct Ctx;

// Stream-ordered device allocation owned by a context.
struct DevBuf {
  Ctx* ctx = nullptr;
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(Ctx* c, size_t b);
  ~DevBuf();
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept { *this = std::move(o); }
  DevBuf& operator=(DevBuf&& o) noexcept;
  uint64_t* u64() const { return static_cast<uint64_t*>(p); }
  void reset();
};

// Basis-conversion tables of one level (ModUp for every digit, ModDown).
struct ConvTables {
  int l = 0, beta = 0, rows = 0;  // rows = l + alpha
  // ModUp: for digit j, local a < alpha: v = [x * Dhat^-1]_{q}; then for
  // target row r: acc += v * [Dhat]_{m_r}.
  DevBuf dhinv, dhinv_s;   // [beta][alpha]
  DevBuf dh, dh_s;         // [beta][alpha][rows]
  DevBuf dhw, dhw_s;       // [beta][alpha][rows]: dh times psi^(N/2) of the row's modulus
  DevBuf ext_pattern;      // int16 [beta*rows]: modulus index of the row, -1 = digit row
  DevBuf pq_pattern;       // int16 [rows]: -1 for Q rows, special modulus for P rows
  DevBuf qp_pattern;       // int16 [rows]: the modulus of every QP_l row (Q limbs, then P)
  DevBuf md_pinv, md_pinv_s;  // [l]: P^-1 mod q_i
  DevBuf xs_post, xs_post_s;  // [l]: N^-1 Dhat_i^-1 mod q_i (fused ModUp)
  DevBuf md_post, md_post_s;  // [rows]: N^-1 Phat_a^-1 mod p_a on P rows (fused ModDown)
  // HMult's merged relinearise + rescale: division by M = P q_level with the
  // dropped moduli D = {q_level, p_0 .. p_{alpha-1}} (rows level .. level+alpha)
  DevBuf rr_pattern;          // int16 [rows]: modulus of the D rows, -1 elsewhere
  DevBuf rr_post, rr_post_s;  // [rows]: N^-1 (M/m)^-1 mod m on the D rows (fused)
  DevBuf rr_yinv, rr_yinv_s;  // [alpha+1]: (M/m)^-1 mod m (unfused)
  DevBuf rr_mh, rr_mh_s;      // [alpha+1][l]: (M/m) mod q_i
  DevBuf rr_minv, rr_minv_s;  // [l]: M^-1 mod q_i
  uint64_t rr_pq = 0, rr_pq_s = 0;  // P mod q_level and its Shoup companion
  // centred conversions: overflow u = floor(sum_m v_m / m + 1/2) in double,
  // then u [M]_{q_i} subtracted (M = P for ModDown, P q_level merged)
  DevBuf md_inv;              // double [alpha]: 1 / p_a
  std::vector<double> md_inv_h, rr_inv_h;  // host copies of md_inv and rr_inv
  DevBuf md_pq, md_pq_s;      // [l]: P mod q_i
  DevBuf rr_inv;              // double [alpha+1]: 1 / q_level, 1 / p_a
  DevBuf rr_mq, rr_mq_s;      // [l]: M mod q_i
};

// Kernel kinds timed by the optional per-launch CUDA-event profiler.
enum KernelKind {
  K_NTT_SMALL, K_NTT_FWD, K_NTT_INV, K_MODUP_NTT, K_MODDOWN_NTT, K_RESCALE_NTT,
  K_MODUP, K_INNER, K_MD_CONV, K_MD_FINISH, K_TENSOR, K_MUL_PT, K_ADD, K_MUL_INT,
  K_LINCOMB, K_ROT_FINISH, K_AUTO, K_RS_SPREAD, K_RS_FINISH, K_INT_RNS, K_ENCODE,
  K_SAMPLE, K_CRYPT, K_COPY, K_RR_NTT, K_RR_TOP, K_OVERFLOW, K_KIND_COUNT
};
const char* kernel_kind_name(int k);

// NTT tuning slots: the clustered transform kernels per descriptor kind
enum NttSlot {
  NTT_SLOT_FWD, NTT_SLOT_MODUP, NTT_SLOT_MODDOWN, NTT_SLOT_RESCALE, NTT_SLOT_RELIN_RESCALE,
  NTT_SLOT_INV, NTT_SLOT_COUNT
};

struct ProfRec {
  int kind;
  double bytes;
  double ops;  // algorithmic 64-bit modular multiplications
  cudaEvent_t a, b;
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int log_n = 0;
  uint64_t N = 0;
  int L = 0, alpha = 0, n_qp = 0, beta_max = 0;
  // fused NTT kernels (basis conversion / rescale inside the transforms'
  // loads and stores); off = separate conversion and transform launches
  bool fused = true;
  // CTAs per SM of the clustered transforms, per tuning slot (1 or 2)
  int ntt_minb[NTT_SLOT_COUNT] = {2, 2, 2, 2, 2, 2};
  std::vector<uint64_t> mod, psi;
  std::vector<double> delta;
  // device tables
  DevBuf d_mod;             // Mod[n_qp]
  DevBuf d_tw, d_tws;       // [n_qp][N] psi^brv(k) and Shoup companions
  DevBuf d_itw, d_itws;     // inverse
  DevBuf d_ninv, d_ninvs;   // [n_qp]
  // radix-8 round twiddles (N >= 8192): per modulus, per round node k of the
  // stage tree, 7 (twiddle, Shoup) pairs: node, its 2 children, 4 grandchildren
  DevBuf d_tw8, d_itw8;
  size_t tw8_nodes = 0;     // nodes per modulus
  DevBuf d_iota;            // int16 [n_qp]: 0..n_qp-1
  DevBuf d_fft;             // double [2N][2]: cos, sin of 2 pi k / 2N
  DevBuf d_slot;            // uint32 [N/2]: k_j = (5^j mod 2N - 1) / 4
  DevBuf d_md_yinv, d_md_yinv_s;  // [alpha]: Phat_a^-1 mod p_a
  DevBuf d_md_ph, d_md_ph_s;      // [alpha][L+1]: Phat_a mod q_i
  std::map<int, std::unique_ptr<ConvTables>> conv;
  std::map<uint64_t, std::unique_ptr<DevBuf>> perms;  // galois -> uint32[N]
  // rescale of k c by q_r: (r, k) -> [N^-1 k mod q_r, Shoup, k q_r^-1 mod q_t (t < r), Shoup]
  std::map<std::pair<int, int64_t>, std::unique_ptr<DevBuf>> scaled;
  const uint64_t* scaled_consts(int r, int64_t k);
  DevBuf d_flag;            // int32 device status words: [0] encoding overflow,
                            // [1] a time-bounded device wait ran out
  unsigned* wait_status() const { return static_cast<unsigned*>(d_flag.p) + 1; }
  void check_waits();       // after a stream synchronize: CKKS_ERR_TIMEOUT if [1] set
  DevBuf d_rs_inv, d_rs_invs;     // [(L+1)][(L+1)]: q_l^-1 mod q_t at [l][t]
  DevBuf d_pmod;                  // [L+1]: P mod q_t

  // launch accounting and optional per-launch event timing
  uint64_t launches[K_KIND_COUNT] = {};
  bool prof = false;
  std::vector<ProfRec> prof_recs;
  // while a schedule is captured into a CUDA graph, its launch records go
  // to the graph's own list (its events become event-record nodes)
  std::vector<ProfRec>* prof_sink = nullptr;
  // per kind, from replayed graphs: ms, algorithmic bytes, modmuls, launches
  double prof_acc[K_KIND_COUNT][4] = {};
  std::vector<cudaEvent_t> ev_pool;
  cudaEvent_t take_event();

  ~Ctx();
  const Mod* dmod() const { return static_cast<const Mod*>(d_mod.p); }
  const int16_t* iota() const { return static_cast<const int16_t*>(d_iota.p); }
  ConvTables& tables(int level);
  const uint32_t* perm(uint64_t galois);
  uint64_t galois(int64_t step) const;
};

}  // namespace ck

// ABI handle types
struct ckks_ctx {
  ck::Ctx c;
};

struct ckks_keys {
  ck::Ctx* ctx;
  ck::DevBuf s;                                   // [n_qp][N] NTT form
  ck::DevBuf relin;                               // [beta_max][2][n_qp][N]
  std::map<uint64_t, std::unique_ptr<ck::DevBuf>> galois;
  // the switching keys' uniform halves come from this public seed (the
  // secret's seed when none was given); seed-compressed keys keep only the
  // b halves ([beta_max][n_qp][N]) and regenerate a from it on use
  uint64_t a_seed = 0;
  bool own_a_seed = false;
  bool compressed = false;
};

struct ckks_ct {
  ck::Ctx* ctx;
  ck::DevBuf d;  // [B][2][level+1][N]
  size_t B;
  int level;
  double scale;
  size_t words() const { return B * 2 * (size_t)(level + 1) * ctx->N; }
};

namespace ck {

// RAII marker around one launch (or copy): counts it and, when profiling is
// on, brackets it with events on the context's stream.
struct Launch {
  Ctx& c;
  int kind;
  double bytes;
  cudaEvent_t b = nullptr;
  Launch(Ctx& cx, int k, double algorithmic_bytes, double modmuls = 0.0);
  ~Launch();
};

// ---- host helpers (context.cu)
uint64_t mulmod_h(uint64_t a, uint64_t b, uint64_t q);
uint64_t powmod_h(uint64_t b, uint64_t e, uint64_t q);
uint64_t invmod_h(uint64_t a, uint64_t q);
uint64_t shoup_h(uint64_t w, uint64_t q);
Mod make_mod(uint64_t q);
bool is_prime_h(uint64_t n);
int gen_chain(int log_n, int q0_bits, int scale_bits, int n_scale, int p_bits, int n_special,
              std::vector<uint64_t>& mod, std::vector<double>& delta);
void ctx_init(Ctx& c, int log_n, int q0_bits, int scale_bits, int n_scale, int p_bits,
              int n_special, int device);

// ---- NTT (ntt.cu): rows r at base + r*N use modulus pattern[r % P]; a
// negative pattern entry skips the row.
// `active` = rows actually transformed (for traffic accounting).
void ntt_forward(Ctx& c, uint64_t* base, size_t n_rows, const int16_t* pattern, int P,
                 size_t active = SIZE_MAX);
void ntt_inverse(Ctx& c, uint64_t* base, size_t n_rows, const int16_t* pattern, int P,
                 size_t active = SIZE_MAX);

// Fused row kernels (N >= 8192): ModUp conversion in the forward NTT's
// loads; ModDown / rescale subtract-and-scale in its stores.
bool ntt_fused_available(const Ctx& c);
// inverse NTT with a per-row post factor (instead of N^-1); out of place
// when src is given (row i of period p read from src + p src_stride + i N)
void ntt_inverse_post(Ctx& c, uint64_t* base, size_t n_rows, const int16_t* pattern, int P,
                      const uint64_t* post, const uint64_t* posts, size_t active = SIZE_MAX,
                      const uint64_t* src = nullptr, size_t src_stride = 0);
void ntt_modup_fused(Ctx& c, const uint64_t* xs, const uint64_t* d, size_t d_stride, size_t B,
                     int level, uint64_t* ext);
// ov: [BK][N] overflow of the centred P -> Q conversion (k_overflow)
void ntt_moddown_fused(Ctx& c, const uint64_t* acc, const uint8_t* ov, size_t BK, int level,
                       uint64_t* out);
void ntt_rescale_fused(Ctx& c, const uint64_t* in, const uint64_t* last, size_t polys, int level,
                       uint64_t* out);
// rescale by q_level of k c (c: poly p at in + p in_stride, limbs 0..level);
// `last` holds the coefficient form of k c_level; kinv[t] = k q_level^-1 mod q_t
void ntt_rescale_scaled_fused(Ctx& c, const uint64_t* in, size_t in_stride, const uint64_t* last,
                              size_t polys, int level, const uint64_t* kinv, const uint64_t* kinvs,
                              uint64_t* out);
// out[B][2][level][N] = (d_k q_level^-1 + (acc_k - Conv_D(acc_D)) M^-1), transformed
void ntt_relin_rescale_fused(Ctx& c, const uint64_t* acc, const uint64_t* d, const uint8_t* ov,
                             size_t B, int level, uint64_t* out);

// ---- elementwise (elementwise.cu). Ciphertext batches are [B][polys][l][N].
void k_add(Ctx& c, const uint64_t* a, const uint64_t* b, uint64_t* out, size_t rows, int l,
           bool sub);
void k_mul_pt(Ctx& c, const uint64_t* a, const uint64_t* pt, uint64_t* out, size_t rows, int l);
void k_add_pt_c0(Ctx& c, const uint64_t* a, const uint64_t* pt, uint64_t* out, size_t B, int l);
void k_tensor(Ctx& c, const uint64_t* a, const uint64_t* b, uint64_t* out, size_t B, int l,
              bool accumulate);
void k_copy_limbs(Ctx& c, const uint64_t* in, int l_in, uint64_t* out, int l_out, size_t polys);
void k_automorphism(Ctx& c, const uint64_t* in, uint64_t* out, size_t rows, const uint32_t* perm);
void k_rescale_spread(Ctx& c, const uint64_t* last, uint64_t* out, size_t polys, int level);
void k_int_to_rns(Ctx& c, const int64_t* v, uint64_t* out, size_t polys, int rows,
                  const int16_t* pattern);

// ---- key switching (keyswitch.cu)
// d: batch element b at d + b d_stride (default l N words), [l][N] NTT;
// ext out: [B][beta][l+alpha][N] NTT.
void modup(Ctx& c, const uint64_t* d, size_t B, int level, uint64_t* ext, size_t d_stride = 0);
// out[B][2][l][N] = ModDown(<sigma_g(ext), key>); galois 0 = no automorphism.
void keyswitch_ext(Ctx& c, const uint64_t* ext, size_t B, int level, const uint64_t* key,
                   uint64_t galois, uint64_t* out);
// HMult's relinearise + rescale in one division by P q_level: d is the tensor
// product [B][3][level+1][N], ext the ModUp of its d2; out [B][2][level][N].
// one CTA whose bounded mbarrier wait runs out (self-test of the status word)
void wait_selftest(Ctx& c, long long limit);
void relin_rescale_ext(Ctx& c, const uint64_t* d, const uint64_t* ext, size_t B, int level,
                       const uint64_t* key, uint64_t* out);
// double-hoisted BSGS: the key inner product of sigma_g(ext) over QP_l
// ([B][2][l + alpha][N], no ModDown), and the division of such a QP_l pair
// by P q_level (its D rows are transformed in place); out [B][2][level][N]
DevBuf keyswitch_qp(Ctx& c, const uint64_t* ext, size_t B, int level, const uint64_t* key,
                    uint64_t galois);
void div_p_ql(Ctx& c, uint64_t* acc, size_t B, int level, uint64_t* out);

// ---- encoding (encode.cu)
// v: device doubles [B][nv]; writes pt [B][level+1][N] at `scale`. Returns
// CKKS_ERR_OVERFLOW if a coefficient does not fit int64.
int encode(Ctx& c, const double* d_v, size_t B, size_t nv, int level, double scale, uint64_t* pt);
// the same integer coefficients reduced mod the moduli pattern[0 .. rows-1]
// (e.g. a QP_l plaintext): pt [B][rows][N], NTT form; d_im (optional):
// the slots' imaginary parts, [B][nv] like d_v
int encode_rows(Ctx& c, const double* d_v, size_t B, size_t nv, int rows, const int16_t* pattern,
                double scale, uint64_t* pt, const double* d_im = nullptr);
// m: [B][N] limb-0 coefficient values (uint64 mod q0); out: device doubles [B][nv]
void decode_limb0(Ctx& c, const uint64_t* m, size_t B, double scale, double* d_out, size_t nv);

// ---- sampling (sample.cu)
void sample_ternary(Ctx& c, uint64_t seed, int64_t* out);
// uniform residues of objects id_base .. id_base + count - 1, object o at
// out + o obj_rows N (rows rows each, moduli pattern[r])
void sample_uniform_seq(Ctx& c, uint64_t seed, uint64_t id_base, size_t count, int rows,
                        const int16_t* pattern, uint64_t* out, size_t obj_rows);
void sample_sparse_ternary(Ctx& c, uint64_t seed, int h, int64_t* out);
void sample_cbd(Ctx& c, uint64_t seed, const uint64_t* ids, size_t count, int64_t* out);
void sample_uniform(Ctx& c, uint64_t seed, const uint64_t* ids, size_t count, int rows,
                    const int16_t* pattern, uint64_t* out);

}  // namespace ck
