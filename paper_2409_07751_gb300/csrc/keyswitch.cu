// Hybrid key switching: ModUp (fast basis conversion per digit), key inner
// product over the extended basis QP (with the Galois automorphism of a
// hoisted rotation fused into its loads), and ModDown.
//
// ModUp of digit j (Q primes D_j = [j*alpha, min((j+1)*alpha, l))):
//   rows in D_j copy the NTT-form input;
//   other rows t: sum_{i in D_j} [x_i Dhat_i^{-1}]_{q_i} (Dhat_i mod m_t) mod m_t,
//   then NTT.
// ModDown: out_i = (acc_i - Conv_{P->Q}([acc]_P)_i) * P^{-1} mod q_i.
#include <algorithm>

#include "modarith.cuh"
#include "tma.cuh"

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

constexpr int MAX_ALPHA = 16;

// thread per (b, j, n); xc: [B][l][N] coefficient form; d: NTT form
__global__ void modup_kernel(const uint64_t* xc, const uint64_t* d, uint64_t* ext, size_t B,
                             int log_n, int l, int alpha, int beta, int rows, int L,
                             const Mod* mods, const uint64_t* dhinv, const uint64_t* dhinvs,
                             const uint64_t* dh, const uint64_t* dhs) {
  const size_t N = (size_t)1 << log_n;
  GRID_LOOP(idx, B * (size_t)beta * N) {
    const size_t n = idx & (N - 1);
    const size_t bj = idx >> log_n;
    const int j = (int)(bj % beta);
    const size_t b = bj / beta;
    const int lo = j * alpha;
    const int hi = min((j + 1) * alpha, l);
    uint64_t v[MAX_ALPHA];
    for (int a = 0; a < hi - lo; a++) {
      const int i = lo + a;
      const uint64_t x = xc[(b * l + i) * N + n];
      v[a] = mul_shoup(x, dhinv[j * alpha + a], dhinvs[j * alpha + a], mods[i].q);
    }
    uint64_t* out = ext + ((b * beta + j) * rows) * N + n;
    for (int r = 0; r < rows; r++) {
      if (r >= lo && r < hi) {
        out[(size_t)r * N] = d[(b * l + r) * N + n];
        continue;
      }
      const int mi = r < l ? r : L + 1 + (r - l);
      const uint64_t m = mods[mi].q;
      uint64_t acc = 0;
      for (int a = 0; a < hi - lo; a++) {
        const size_t ti = ((size_t)(j * alpha + a)) * rows + r;
        acc = add_mod(acc, mul_shoup(v[a], dh[ti], dhs[ti], m), m);
      }
      out[(size_t)r * N] = acc;
    }
  }
}

constexpr int IP_THREADS = 128;

template <int NB, class F>
__device__ __forceinline__ void for_digits(int beta, F body) {
  if constexpr (NB > 0) {
#pragma unroll
    for (int j = 0; j < NB; j++) body(j);
  } else {
    for (int j = 0; j < beta; j++) body(j);
  }
}

// The two outputs (key halves h = 0, 1) of one coefficient of the key inner
// product: o_h = sum_j e_j k_{j,h} mod m over the beta digits. e_at(j) and
// k_at(j, h) fetch the operands. Moduli of 33..48 bits sum 32-bit partial
// products apart and reduce once; wider moduli sum 128-bit products;
// narrower ones reduce every product. NB > 0: the digit count is the
// compile-time NB (loops unrolled).
template <int NB = 0, class EF, class KF>
__device__ __forceinline__ void ip_point(EF e_at, KF k_at, int beta, const Mod& m, uint64_t& o0,
                                         uint64_t& o1) {
  const bool lazy = m.s >= 33;
  const bool split = lazy && m.s <= 48;
  if (split) {
    // e, k < 2^48: e k = e0 k0 + (e0 k1 + e1 k0) 2^32 + e1 k1 2^64 with
    // 16-bit e1, k1; the partial products are summed apart (the halves
    // of e0 k0 separately, so no sum carries) and combined once
    uint64_t a0[2] = {0, 0}, a1[2] = {0, 0}, bm[2] = {0, 0}, cc[2] = {0, 0};
    for_digits<NB>(beta, [&](int j) {
      const uint64_t e = e_at(j);
      const uint32_t el = (uint32_t)e, eh = (uint32_t)(e >> 32);
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const uint64_t k = k_at(j, h);
        const uint32_t kl = (uint32_t)k, kh = (uint32_t)(k >> 32);
        const uint64_t p = (uint64_t)el * kl;
        a0[h] += (uint32_t)p;
        a1[h] += p >> 32;
        bm[h] += (uint64_t)el * kh + (uint64_t)eh * kl;
        cc[h] += (uint64_t)eh * kh;
      }
    });
    // the sum x = hi 2^64 + lo has hi < 2^37 (beta <= 32 products below
    // 2^96), so x' = hi [2^64]_m + lo < 2^64 + 2^85 is below 2^(2s) for
    // s = 33 .. 48 and one Barrett reduction gives x mod m
    uint64_t o[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const uint64_t mid = a1[h] + bm[h];
      const uint64_t lo = a0[h] + (mid << 32);
      const uint64_t hi = cc[h] + (mid >> 32) + (lo < a0[h] ? 1 : 0);
      const uint64_t plo = hi * m.t64, phi = __umul64hi(hi, m.t64);
      const uint64_t slo = plo + lo;
      o[h] = reduce128(slo, phi + (slo < plo ? 1 : 0), m);
    }
    o0 = o[0];
    o1 = o[1];
  } else if (lazy) {
    uint64_t l0 = 0, h0 = 0, l1 = 0, h1 = 0;
    for_digits<NB>(beta, [&](int j) {
      const uint64_t e = e_at(j);
      const uint64_t k0 = k_at(j, 0), k1 = k_at(j, 1);
      uint64_t p = e * k0;
      h0 += __umul64hi(e, k0) + ((l0 + p) < l0 ? 1 : 0);
      l0 += p;
      p = e * k1;
      h1 += __umul64hi(e, k1) + ((l1 + p) < l1 ? 1 : 0);
      l1 += p;
    });
    o0 = reduce_wide(l0, h0, m);
    o1 = reduce_wide(l1, h1, m);
  } else {
    uint64_t a0 = 0, a1 = 0;
    for_digits<NB>(beta, [&](int j) {
      const uint64_t e = e_at(j);
      a0 = add_mod(a0, mul_mod(e, k_at(j, 0), m), m.q);
      a1 = add_mod(a1, mul_mod(e, k_at(j, 1), m), m.q);
    });
    o0 = a0;
    o1 = a1;
  }
}

// thread per (r, n); loops over the batch so each key word is read from HBM
// once per launch. The thread's 2*beta key words sit in shared memory (a
// private slice per thread, so no synchronization). Used when fusion is off
// or an operand is not 16-byte aligned.
// ext: [B][beta][rows][N]; key: [beta_max][2][n_qp][N]; acc: [B][2][rows][N]
__global__ void __launch_bounds__(IP_THREADS)
    inner_product_kernel(const uint64_t* ext, const uint64_t* key, uint64_t* acc, size_t B,
                         int log_n, int l, int beta, int rows, int L, int n_qp, const Mod* mods,
                         const uint32_t* perm) {
  extern __shared__ uint64_t kw[];  // [2*beta][IP_THREADS]
  const size_t N = (size_t)1 << log_n;
  const uint32_t tid = threadIdx.x;
  GRID_LOOP(idx, (size_t)rows * N) {
    const size_t n = idx & (N - 1);
    const int r = (int)(idx >> log_n);
    const int mi = r < l ? r : L + 1 + (r - l);
    const Mod m = mods[mi];
    const size_t src = perm ? perm[n] : n;
    for (int j = 0; j < beta; j++) {
      kw[(2 * j) * IP_THREADS + tid] = key[(((size_t)j * 2 + 0) * n_qp + mi) * N + n];
      kw[(2 * j + 1) * IP_THREADS + tid] = key[(((size_t)j * 2 + 1) * n_qp + mi) * N + n];
    }
    for (size_t b = 0; b < B; b++) {
      const uint64_t* e0 = ext + ((b * beta) * rows + r) * N + src;
      uint64_t o0, o1;
      ip_point([&](int j) { return e0[(size_t)j * rows * N]; },
               [&](int j, int h) { return kw[(2 * j + h) * IP_THREADS + tid]; }, beta, m, o0, o1);
      acc[((b * 2 + 0) * rows + r) * N + n] = o0;
      acc[((b * 2 + 1) * rows + r) * N + n] = o1;
    }
  }
}

// TMA-staged key inner product. One CTA per (row r, tile of T consecutive
// coefficients), one thread per coefficient. Thread 0 stages the tile's
// 2 beta key words by bulk copies once, then streams the batch: the beta
// extension tiles of element b land in stage b % S (S stages in flight),
// each stage completed on its own mbarrier. With a Galois automorphism the
// T outputs of an aligned tile read an aligned tile of T sources (the NTT
// -domain permutation only permutes the low log2 T index bits, checked when
// the table is built), so the copies stay contiguous.
// smem: keys [2 beta][T], then [S][beta][T].
// BETA > 0 (digit counts up to IP_REG_BETA): the thread's key words move
// from shared memory into registers once, and the digit loops unroll.
constexpr int IP_TMA_MAX_T = 256;
constexpr int IP_TMA_MAX_STAGES = 4;
constexpr int IP_REG_BETA = 8;

template <int BETA>
__global__ void __launch_bounds__(IP_TMA_MAX_T, 2)
    inner_product_tma(const uint64_t* ext, const uint64_t* key, uint64_t* acc, int B, int log_n,
                      int l, int beta, int rows, int L, int n_qp, const Mod* mods,
                      const uint32_t* perm, int stages, long long limit, unsigned* status) {
  extern __shared__ __align__(128) uint64_t ipsm[];
  __shared__ __align__(8) uint64_t bars[1 + IP_TMA_MAX_STAGES];
  const int T = blockDim.x;
  const size_t N = (size_t)1 << log_n;
  const size_t tiles = N / (size_t)T;
  const int r = (int)(blockIdx.x / tiles);
  const size_t n0 = (blockIdx.x % tiles) * (size_t)T;
  const int tid = threadIdx.x;
  const size_t n = n0 + tid;
  const int mi = r < l ? r : L + 1 + (r - l);
  const size_t src0 = perm ? (perm[n0] & ~(uint32_t)(T - 1)) : n0;
  const int sidx = perm ? (int)(perm[n] - src0) : tid;
  uint64_t* kw = ipsm;                            // [2 beta][T]
  uint64_t* xs = ipsm + (size_t)2 * beta * T;     // [S][beta][T]
  const uint32_t tile = (uint32_t)T * 8u;
  const uint32_t kbar = smem_addr(&bars[0]);
  auto stage_bar = [&](int s) { return smem_addr(&bars[1 + s]); };
  auto issue = [&](int b) {  // thread 0: element b's beta tiles into stage b % S
    const int s = b % stages;
    mbar_expect_tx(stage_bar(s), (uint32_t)beta * tile);
    for (int j = 0; j < beta; j++)
      bulk_load(smem_addr(xs + ((size_t)s * beta + j) * T),
                ext + (((size_t)b * beta + j) * rows + r) * N + src0, tile, stage_bar(s));
  };
  // on a timed-out wait: thread 0 waits (bounded) for every copy still in
  // flight into this CTA's shared memory, records the failure, and the CTA
  // returns with its outputs unwritten
  auto drain = [&](bool keys_pending, int b_first) {
    if (tid != 0) return;
    if (keys_pending) mbar_wait(kbar, 0, limit);
    for (int b = b_first; b < B && b < b_first + stages; b++)
      mbar_wait(stage_bar(b % stages), (uint32_t)(b / stages) & 1u, limit);
    atomicOr(status, 1u);
  };
  if (tid == 0) {
    mbar_init(kbar, 1);
    for (int s = 0; s < stages; s++) mbar_init(stage_bar(s), 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (tid == 0) {
    mbar_expect_tx(kbar, 2u * (uint32_t)beta * tile);
    for (int j = 0; j < beta; j++)
      for (int h = 0; h < 2; h++)
        bulk_load(smem_addr(kw + (size_t)(2 * j + h) * T),
                  key + (((size_t)j * 2 + h) * n_qp + mi) * N + n0, tile, kbar);
    for (int b = 0; b < B && b < stages; b++) issue(b);
  }
  const Mod m = mods[mi];
  if (__syncthreads_or(!mbar_wait(kbar, 0, limit))) {
    drain(true, 0);
    return;
  }
  uint64_t kr[2 * (BETA > 0 ? BETA : 1)];
  if constexpr (BETA > 0) {
#pragma unroll
    for (int i = 0; i < 2 * BETA; i++) kr[i] = kw[(size_t)i * T + tid];
  }
  for (int b = 0; b < B; b++) {
    const int s = b % stages;
    if (__syncthreads_or(!mbar_wait(stage_bar(s), (uint32_t)(b / stages) & 1u, limit))) {
      drain(false, b);
      return;
    }
    const uint64_t* x = xs + (size_t)s * beta * T + sidx;
    uint64_t o0, o1;
    if constexpr (BETA > 0)
      ip_point<BETA>([&](int j) { return x[(size_t)j * T]; },
                     [&](int j, int h) { return kr[2 * j + h]; }, beta, m, o0, o1);
    else
      ip_point([&](int j) { return x[(size_t)j * T]; },
               [&](int j, int h) { return kw[(size_t)(2 * j + h) * T + tid]; }, beta, m, o0,
               o1);
    acc[(((size_t)b * 2 + 0) * rows + r) * N + n] = o0;
    acc[(((size_t)b * 2 + 1) * rows + r) * N + n] = o1;
    __syncthreads();  // stage s fully read before it is refilled
    if (tid == 0 && b + stages < B) issue(b + stages);
  }
}

// an mbarrier phase that no arrival or copy completes: the bounded wait runs
// out and is reported like a stalled staged copy
__global__ void wait_selftest_kernel(long long limit, unsigned* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_addr(&bar), 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (__syncthreads_or(!mbar_wait(smem_addr(&bar), 0, limit)) && threadIdx.x == 0)
    atomicOr(status, 1u);
}

// overflow of the centred conversion, u = floor(sum_m v_m inv_m + 1/2) in
// double precision, m ascending, no contraction (the oracle's expression)
__device__ __forceinline__ uint64_t conv_overflow(const uint64_t* v, const double* inv, int n) {
  double sf = 0.0;
  for (int m = 0; m < n; m++) sf = __dadd_rn(sf, __dmul_rn(__ull2double_rn(v[m]), inv[m]));
  return (uint64_t)floor(sf + 0.5);
}

// thread per (bk, n): y_a = [acc_P[a] Phat_a^{-1}]_{p_a};
// conv_i = sum_a y_a Phat_a - u P mod q_i (centred conversion)
__global__ void moddown_conv_kernel(const uint64_t* acc, uint64_t* conv, size_t BK, int log_n,
                                    int l, int alpha, int rows, int L, const Mod* mods,
                                    const uint64_t* yinv, const uint64_t* yinvs,
                                    const uint64_t* ph, const uint64_t* phs, const double* inv,
                                    const uint64_t* pq, const uint64_t* pqs) {
  const size_t N = (size_t)1 << log_n;
  GRID_LOOP(idx, BK * N) {
    const size_t n = idx & (N - 1);
    const size_t bk = idx >> log_n;
    uint64_t y[MAX_ALPHA];
    for (int a = 0; a < alpha; a++) {
      const uint64_t x = acc[(bk * rows + l + a) * N + n];
      y[a] = mul_shoup(x, yinv[a], yinvs[a], mods[L + 1 + a].q);
    }
    const uint64_t u = conv_overflow(y, inv, alpha);
    for (int i = 0; i < l; i++) {
      const uint64_t q = mods[i].q;
      uint64_t s = 0;
      for (int a = 0; a < alpha; a++) {
        const size_t ti = (size_t)a * (L + 1) + i;
        s = add_mod(s, mul_shoup(y[a], ph[ti], phs[ti], q), q);
      }
      conv[(bk * l + i) * N + n] = sub_mod(s, mul_shoup(u, pq[i], pqs[i], q), q);
    }
  }
}

// The same u, decided in single precision wherever that is certain. Each
// term v_m / m < 1 is within 3.0001 u of its float product (u = 2^-24: the
// conversions of v_m and 1/m and the product), the running sums of at most
// 17 terms (partial sums below 17) add at most 152 u, and t = s + 1/2 one
// more rounding below 18 u: |t - (S + 1/2)| < 221 u < 1.4e-5 for the exact
// S = sum_m v_m / m. When the fraction of t is more than 2^-10 from an
// integer, floor(t) = floor(S + 1/2) = the double expression's result (that
// one is within 1e-13 of S + 1/2); otherwise the double expression decides.
struct InvF {
  float v[MAX_ALPHA + 1];  // float(1 / m)
};
__device__ __forceinline__ uint64_t conv_overflow_fast(const uint64_t* v, const double* inv,
                                                       const InvF& invf, int n) {
  float s = 0.0f;
  for (int m = 0; m < n; m++) s = __fadd_rn(s, __fmul_rn(__ull2float_rn(v[m]), invf.v[m]));
  const float t = __fadd_rn(s, 0.5f);
  const float f = floorf(t);
  const float fr = t - f;  // exact (Sterbenz)
  if (fr > 0x1p-10f && fr < 1.0f - 0x1p-10f) return (uint64_t)f;
  return conv_overflow(v, inv, n);
}

// fused paths: u per (bk, n) from `count` rows starting at `first`, which
// already hold v_m (inverse-transformed and scaled by (M/m)^-1)
__global__ void overflow_kernel(const uint64_t* acc, uint8_t* ov, size_t BK, int log_n, int first,
                                int count, int rows, const double* inv, InvF invf) {
  const size_t N = (size_t)1 << log_n;
  GRID_LOOP(idx, BK * N) {
    const size_t n = idx & (N - 1);
    const size_t bk = idx >> log_n;
    uint64_t v[MAX_ALPHA + 1];
    for (int m = 0; m < count; m++) v[m] = acc[(bk * rows + first + m) * N + n];
    ov[idx] = (uint8_t)conv_overflow_fast(v, inv, invf, count);
  }
}

InvF inv_float(const std::vector<double>& inv) {
  InvF f{};
  for (size_t m = 0; m < inv.size() && m < (size_t)(MAX_ALPHA + 1); m++) f.v[m] = (float)inv[m];
  return f;
}

__global__ void moddown_finish_kernel(const uint64_t* acc, const uint64_t* conv, uint64_t* out,
                                      size_t BK, int log_n, int l, int rows, const Mod* mods,
                                      const uint64_t* pinv, const uint64_t* pinvs) {
  const size_t N = (size_t)1 << log_n;
  GRID_LOOP(idx, BK * l * N) {
    const size_t n = idx & (N - 1);
    const size_t bi = idx >> log_n;
    const int i = (int)(bi % l);
    const size_t bk = bi / l;
    const uint64_t q = mods[i].q;
    const uint64_t a = acc[(bk * rows + i) * N + n];
    out[idx] = mul_shoup(sub_mod(a, conv[idx], q), pinv[i], pinvs[i], q);
  }
}

// merged relinearise + rescale: acc row `level` of (b, k) += [P]_{q_level} d_k[level]
__global__ void rr_top_kernel(uint64_t* acc, const uint64_t* d, size_t B, int log_n, int level,
                              int rows, uint64_t q, uint64_t pq, uint64_t pqs) {
  const size_t N = (size_t)1 << log_n;
  const int l = level + 1;
  GRID_LOOP(idx, B * 2 * N) {
    const size_t n = idx & (N - 1);
    const size_t bk = idx >> log_n;
    const size_t b = bk / 2, k = bk % 2;
    uint64_t* a = acc + (bk * rows + level) * N + n;
    *a = add_mod(mul_shoup(d[((b * 3 + k) * l + level) * N + n], pq, pqs, q), *a, q);
  }
}

// unfused: thread per (bk, n): y_m = [acc_m (M/m)^-1]_m over the D rows
// (coefficient form), conv_i = sum_m y_m [M/m]_{q_i} - u [M]_{q_i}, i < level
__global__ void rr_conv_kernel(const uint64_t* acc, uint64_t* conv, size_t BK, int log_n,
                               int level, int alpha, int rows, const Mod* mods, const int16_t* dmod,
                               const uint64_t* yinv, const uint64_t* yinvs, const uint64_t* mh,
                               const uint64_t* mhs, const double* inv, const uint64_t* mq,
                               const uint64_t* mqs) {
  const size_t N = (size_t)1 << log_n;
  const int l = level + 1;
  GRID_LOOP(idx, BK * N) {
    const size_t n = idx & (N - 1);
    const size_t bk = idx >> log_n;
    uint64_t y[MAX_ALPHA + 1];
    for (int m = 0; m <= alpha; m++) {
      const uint64_t x = acc[(bk * rows + level + m) * N + n];
      y[m] = mul_shoup(x, yinv[m], yinvs[m], mods[dmod[level + m]].q);
    }
    const uint64_t u = conv_overflow(y, inv, alpha + 1);
    for (int i = 0; i < level; i++) {
      const uint64_t q = mods[i].q;
      uint64_t s = 0;
      for (int m = 0; m <= alpha; m++) {
        const size_t ti = (size_t)m * l + i;
        s = add_mod(s, mul_shoup(y[m], mh[ti], mhs[ti], q), q);
      }
      conv[(bk * level + i) * N + n] = sub_mod(s, mul_shoup(u, mq[i], mqs[i], q), q);
    }
  }
}

// unfused: out_k[i] = d_k[i] q_level^-1 + (acc_k[i] - conv_i) M^-1
__global__ void rr_finish_kernel(const uint64_t* acc, const uint64_t* d, const uint64_t* conv,
                                 uint64_t* out, size_t BK, int log_n, int level, int rows,
                                 const Mod* mods, const uint64_t* minv, const uint64_t* minvs,
                                 const uint64_t* qlinv, const uint64_t* qlinvs) {
  const size_t N = (size_t)1 << log_n;
  const int l = level + 1;
  GRID_LOOP(idx, BK * level * N) {
    const size_t n = idx & (N - 1);
    const size_t bi = idx >> log_n;
    const int i = (int)(bi % level);
    const size_t bk = bi / level;
    const size_t b = bk / 2, k = bk % 2;
    const uint64_t q = mods[i].q;
    const uint64_t a = acc[(bk * rows + i) * N + n];
    const uint64_t r = mul_shoup(sub_mod(a, conv[idx], q), minv[i], minvs[i], q);
    if (!d) {
      out[idx] = r;
      continue;
    }
    const uint64_t dv = d[((b * 3 + k) * l + i) * N + n];
    out[idx] = add_mod(mul_shoup(dv, qlinv[i], qlinvs[i], q), r, q);
  }
}

}  // namespace

void modup(Ctx& c, const uint64_t* d, size_t B, int level, uint64_t* ext, size_t d_stride) {
  ConvTables& T = c.tables(level);
  const int l = T.l;
  if (c.alpha > MAX_ALPHA) throw Error(CKKS_ERR_UNSUPPORTED, "alpha > 16");
  if (d_stride == 0) d_stride = (size_t)l * c.N;
  DevBuf xc(&c, B * l * c.N * 8);
  if (ntt_fused_available(c)) {
    // the inverse transform reads d in place and writes the scaled coefficients to xc
    ntt_inverse_post(c, xc.u64(), B * l, c.iota(), l, T.xs_post.u64(), T.xs_post_s.u64(), SIZE_MAX,
                     d, d_stride);
    ntt_modup_fused(c, xc.u64(), d, d_stride, B, level, ext);
    return;
  }
  {
    Launch L_(c, K_COPY, 2.0 * (double)xc.bytes);
    CK_CUDA(cudaMemcpy2DAsync(xc.p, (size_t)l * c.N * 8, d, d_stride * 8, (size_t)l * c.N * 8, B,
                              cudaMemcpyDeviceToDevice, c.stream));
  }
  DevBuf dc;  // the unfused kernel reads d densely
  const uint64_t* dd = d;
  if (d_stride != (size_t)l * c.N) {
    dc = DevBuf(&c, B * l * c.N * 8);
    Launch L_(c, K_COPY, 2.0 * (double)dc.bytes);
    CK_CUDA(cudaMemcpy2DAsync(dc.p, (size_t)l * c.N * 8, d, d_stride * 8, (size_t)l * c.N * 8, B,
                              cudaMemcpyDeviceToDevice, c.stream));
    dd = dc.u64();
  }
  ntt_inverse(c, xc.u64(), B * l, c.iota(), l);
  const double W8 = (double)c.N * 8.0;
  {
  Launch L_(c, K_MODUP, W8 * (double)B * (2.0 * l + (double)T.beta * T.rows));
  modup_kernel<<<grid_for(B * T.beta * c.N), TPB, 0, c.stream>>>(
      xc.u64(), dd, ext, B, c.log_n, l, c.alpha, T.beta, T.rows, c.L, c.dmod(), T.dhinv.u64(),
      T.dhinv_s.u64(), T.dh.u64(), T.dh_s.u64());
  CK_CUDA(cudaGetLastError());
  }
  ntt_forward(c, ext, B * T.beta * T.rows, static_cast<const int16_t*>(T.ext_pattern.p),
              T.beta * T.rows, B * ((size_t)T.beta * T.rows - l));
}

// acc[B][2][rows][N] = <sigma_g(ext), key> over QP_l
static DevBuf key_product(Ctx& c, const uint64_t* ext, size_t B, int level, const uint64_t* key,
                          uint64_t galois) {
  ConvTables& T = c.tables(level);
  const int l = T.l, rows = T.rows;
  if (T.beta > MAX_DIGITS) throw Error(CKKS_ERR_UNSUPPORTED, "more than 32 digits");
  const uint32_t* perm = galois ? c.perm(galois) : nullptr;
  DevBuf acc(&c, B * 2 * rows * c.N * 8);
  const double W8 = (double)c.N * 8.0;
  Launch L_(c, K_INNER, W8 * rows * ((double)B * T.beta + 2.0 * T.beta + 2.0 * B),
            2.0 * (double)B * T.beta * rows * (double)c.N);
  const bool aligned = ((reinterpret_cast<uintptr_t>(ext) | reinterpret_cast<uintptr_t>(key) |
                         reinterpret_cast<uintptr_t>(acc.p)) & 15) == 0;
  if (c.fused && aligned && c.N >= 16 && B <= (size_t)INT32_MAX) {
    // tile width T and stage count S: two CTAs per SM within 227 KiB
    const int S = (int)std::min<size_t>(3, B);
    size_t Tw = std::min<size_t>(IP_TMA_MAX_T, c.N);
    while (Tw > 16 && (size_t)(2 + S) * T.beta * Tw * 8 > 110 * 1024) Tw /= 2;
    const size_t smem = (size_t)(2 + S) * T.beta * Tw * 8;
    const size_t blocks = (size_t)rows * (c.N / Tw);
    auto go = [&](auto kernel) {
      CK_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   110 * 1024));
      kernel<<<(unsigned)blocks, (unsigned)Tw, smem, c.stream>>>(
          ext, key, acc.u64(), (int)B, c.log_n, l, T.beta, rows, c.L, c.n_qp, c.dmod(), perm, S,
          WAIT_LIMIT_CYCLES, c.wait_status());
    };
    switch (T.beta) {
      case 1: go(inner_product_tma<1>); break;
      case 2: go(inner_product_tma<2>); break;
      case 3: go(inner_product_tma<3>); break;
      case 4: go(inner_product_tma<4>); break;
      case 5: go(inner_product_tma<5>); break;
      case 6: go(inner_product_tma<6>); break;
      case 7: go(inner_product_tma<7>); break;
      case 8: go(inner_product_tma<8>); break;
      default: go(inner_product_tma<0>); break;
    }
    static_assert(IP_REG_BETA == 8, "dispatch covers digit counts 1 .. 8");
    CK_CUDA(cudaGetLastError());
    return acc;
  }
  const size_t ip_total = (size_t)rows * c.N;
  const size_t ip_blocks = std::min<size_t>((ip_total + IP_THREADS - 1) / IP_THREADS, 152 * 64);
  inner_product_kernel<<<(unsigned)ip_blocks, IP_THREADS, 2 * T.beta * IP_THREADS * 8, c.stream>>>(
      ext, key, acc.u64(), B, c.log_n, l, T.beta, rows, c.L, c.n_qp, c.dmod(), perm);
  CK_CUDA(cudaGetLastError());
  return acc;
}

void wait_selftest(Ctx& c, long long limit) {
  wait_selftest_kernel<<<1, 32, 0, c.stream>>>(limit, c.wait_status());
  CK_CUDA(cudaGetLastError());
}

// Division of y = P d + acc over QP_l by M = P q_level (d may be null: y = acc)
// with the centred conversion of the dropped limbs; acc's D rows are
// transformed in place.
static void div_p_ql_impl(Ctx& c, uint64_t* acc, const uint64_t* d, size_t B, int level,
                          uint64_t* out) {
  ConvTables& T = c.tables(level);
  const int rows = T.rows;
  const double W8 = (double)c.N * 8.0;
  const int16_t* pat = static_cast<const int16_t*>(T.rr_pattern.p);
  const size_t active = B * 2 * (size_t)(c.alpha + 1);
  if (ntt_fused_available(c)) {
    ntt_inverse_post(c, acc, B * 2 * rows, pat, rows, T.rr_post.u64(), T.rr_post_s.u64(), active);
    DevBuf ov(&c, B * 2 * c.N);
    {
      Launch L_(c, K_OVERFLOW, W8 * B * 2.0 * (c.alpha + 1.0) + B * 2.0 * c.N);
      overflow_kernel<<<grid_for(B * 2 * c.N), TPB, 0, c.stream>>>(
          acc, static_cast<uint8_t*>(ov.p), B * 2, c.log_n, level, c.alpha + 1, rows,
          static_cast<const double*>(T.rr_inv.p), inv_float(T.rr_inv_h));
      CK_CUDA(cudaGetLastError());
    }
    ntt_relin_rescale_fused(c, acc, d, static_cast<const uint8_t*>(ov.p), B, level, out);
    return;
  }
  ntt_inverse(c, acc, B * 2 * rows, pat, rows, active);
  DevBuf conv(&c, B * 2 * (size_t)level * c.N * 8);
  {
    Launch L_(c, K_MD_CONV, W8 * B * 2.0 * (c.alpha + 1.0 + level));
    rr_conv_kernel<<<grid_for(B * 2 * c.N), TPB, 0, c.stream>>>(
        acc, conv.u64(), B * 2, c.log_n, level, c.alpha, rows, c.dmod(), pat, T.rr_yinv.u64(),
        T.rr_yinv_s.u64(), T.rr_mh.u64(), T.rr_mh_s.u64(), static_cast<const double*>(T.rr_inv.p),
        T.rr_mq.u64(), T.rr_mq_s.u64());
    CK_CUDA(cudaGetLastError());
  }
  ntt_forward(c, conv.u64(), B * 2 * (size_t)level, c.iota(), level);
  Launch L2_(c, K_MD_FINISH, W8 * B * 2.0 * ((d ? 4.0 : 3.0) * level));
  rr_finish_kernel<<<grid_for(B * 2 * (size_t)level * c.N), TPB, 0, c.stream>>>(
      acc, d, conv.u64(), out, B * 2, c.log_n, level, rows, c.dmod(), T.rr_minv.u64(),
      T.rr_minv_s.u64(), c.d_rs_inv.u64() + (size_t)level * (c.L + 1),
      c.d_rs_invs.u64() + (size_t)level * (c.L + 1));
  CK_CUDA(cudaGetLastError());
}

void relin_rescale_ext(Ctx& c, const uint64_t* d, const uint64_t* ext, size_t B, int level,
                       const uint64_t* key, uint64_t* out) {
  if (level < 1) throw Error(CKKS_ERR_LEVEL, "level exhausted");
  if (c.alpha + 1 > MAX_ALPHA + 1) throw Error(CKKS_ERR_UNSUPPORTED, "alpha > 16");
  ConvTables& T = c.tables(level);
  const int rows = T.rows;
  DevBuf acc = key_product(c, ext, B, level, key, 0);
  const double W8 = (double)c.N * 8.0;
  {
    Launch L_(c, K_RR_TOP, W8 * 2.0 * B * 3.0, 2.0 * B * (double)c.N);
    rr_top_kernel<<<grid_for(B * 2 * c.N), TPB, 0, c.stream>>>(
        acc.u64(), d, B, c.log_n, level, rows, c.mod[level], T.rr_pq, T.rr_pq_s);
    CK_CUDA(cudaGetLastError());
  }
  div_p_ql_impl(c, acc.u64(), d, B, level, out);
}

DevBuf keyswitch_qp(Ctx& c, const uint64_t* ext, size_t B, int level, const uint64_t* key,
                    uint64_t galois) {
  return key_product(c, ext, B, level, key, galois);
}

void div_p_ql(Ctx& c, uint64_t* acc, size_t B, int level, uint64_t* out) {
  if (level < 1) throw Error(CKKS_ERR_LEVEL, "level exhausted");
  if (c.alpha + 1 > MAX_ALPHA + 1) throw Error(CKKS_ERR_UNSUPPORTED, "alpha > 16");
  div_p_ql_impl(c, acc, nullptr, B, level, out);
}

void keyswitch_ext(Ctx& c, const uint64_t* ext, size_t B, int level, const uint64_t* key,
                   uint64_t galois, uint64_t* out) {
  ConvTables& T = c.tables(level);
  const int l = T.l, rows = T.rows;
  DevBuf acc = key_product(c, ext, B, level, key, galois);
  const double W8 = (double)c.N * 8.0;
  if (ntt_fused_available(c)) {
    ntt_inverse_post(c, acc.u64(), B * 2 * rows, static_cast<const int16_t*>(T.pq_pattern.p), rows,
                     T.md_post.u64(), T.md_post_s.u64(), B * 2 * (size_t)c.alpha);
    DevBuf ov(&c, B * 2 * c.N);
    {
      Launch L_(c, K_OVERFLOW, W8 * B * 2.0 * c.alpha + B * 2.0 * c.N);
      overflow_kernel<<<grid_for(B * 2 * c.N), TPB, 0, c.stream>>>(
          acc.u64(), static_cast<uint8_t*>(ov.p), B * 2, c.log_n, l, c.alpha, rows,
          static_cast<const double*>(T.md_inv.p), inv_float(T.md_inv_h));
      CK_CUDA(cudaGetLastError());
    }
    ntt_moddown_fused(c, acc.u64(), static_cast<const uint8_t*>(ov.p), B * 2, level, out);
    return;
  }
  ntt_inverse(c, acc.u64(), B * 2 * rows, static_cast<const int16_t*>(T.pq_pattern.p), rows,
              B * 2 * (size_t)c.alpha);
  DevBuf conv(&c, B * 2 * l * c.N * 8);
  {
  Launch L_(c, K_MD_CONV, W8 * B * 2.0 * (c.alpha + l));
  moddown_conv_kernel<<<grid_for(B * 2 * c.N), TPB, 0, c.stream>>>(
      acc.u64(), conv.u64(), B * 2, c.log_n, l, c.alpha, rows, c.L, c.dmod(), c.d_md_yinv.u64(),
      c.d_md_yinv_s.u64(), c.d_md_ph.u64(), c.d_md_ph_s.u64(),
      static_cast<const double*>(T.md_inv.p), T.md_pq.u64(), T.md_pq_s.u64());
  CK_CUDA(cudaGetLastError());
  }
  ntt_forward(c, conv.u64(), B * 2 * l, c.iota(), l);
  Launch L2_(c, K_MD_FINISH, W8 * B * 2.0 * 3.0 * l);
  moddown_finish_kernel<<<grid_for(B * 2 * l * c.N), TPB, 0, c.stream>>>(
      acc.u64(), conv.u64(), out, B * 2, c.log_n, l, rows, c.dmod(), T.md_pinv.u64(),
      T.md_pinv_s.u64());
  CK_CUDA(cudaGetLastError());
}

}  // namespace ck
