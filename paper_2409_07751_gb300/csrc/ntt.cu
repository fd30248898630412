// Batched negacyclic NTT / inverse NTT over uint64 residues.
//
// Forward map (bit-reversed output): A[j] = sum_i a[i] psi^((2 brv(j)+1) i),
// computed by radix-2 Cooley-Tukey stages m = 1, 2, ..., N/2 where block i
// of stage m uses the twiddle psi^brv(m+i) (the psi twist merged into the
// twiddles). The inverse runs Gentleman-Sande stages m = N/2, ..., 1 with
// psi^-brv(m+i), then scales by N^-1.
//
// N <= 4096: one CTA holds a row in shared memory (radix-2 stages).
// N >= 8192: one CTA per row (limb). N = N1 * N2 with N2 = 4096. The first
// log2(N1) forward stages only couple the elements c + s*N2 (s < N1) of one
// column c, so each thread transforms whole columns in registers and writes
// them back; the CTA's row (<= 512 KiB) stays in L2 between the phases, so
// DRAM sees one read and one write per row. The remaining 12 stages stay
// inside contiguous chunks of N2 elements, transformed in shared memory by
// four radix-8 rounds (three stages per round on 8 elements per thread).
// Butterflies are Harvey's lazy forms: values live in [0, 4q) (forward) or
// [0, 2q) (inverse) and are fully reduced only on the final store.
#include <algorithm>
#include <type_traits>

#include <cooperative_groups.h>

#include "modarith.cuh"

namespace ck {

namespace cg = cooperative_groups;

namespace {

constexpr int CHUNK_LOG = 12;
constexpr int CHUNK = 1 << CHUNK_LOG;  // N2
constexpr int ROW_THREADS = 512;       // one radix-8 group of each of two chunks per thread

// CTAs per cluster (one row per cluster): two chunks (64 KiB of shared
// memory) per CTA and at most 64 registers per thread, so two CTAs share an SM.
template <int N1>
__host__ __device__ constexpr int fwd_cs() { return N1 >= 4 ? N1 / 2 : 1; }
template <int N1>
__host__ __device__ constexpr int inv_cs() { return N1 >= 4 ? N1 / 2 : 1; }
// CTAs per SM the clustered kernels are compiled for: 2 (64 registers per
// thread, 32 warps per SM) by default; 1 (up to 128 registers, no spills in
// the fused descriptors, 16 warps) per tuning slot for N1 >= 8, chosen by
// ckks_autotune_ntt or ckks_set_ntt_shape (Ctx::ntt_minb).
constexpr int CTAS_PER_SM = 2;

// 32-bit address of this CTA's shared-memory location p in the cluster window
// of CTA `rank` (a register instead of a 64-bit generic pointer per peer)
__device__ __forceinline__ uint32_t dsmem_addr(const void* p, uint32_t rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t r;
  asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ uint64_t ld_dsmem(uint32_t addr) {
  uint64_t v;
  asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void st_dsmem(uint32_t addr, uint64_t v) {
  asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t shoup_lazy(uint64_t a, uint64_t w, uint64_t ws, uint64_t q) {
  return mul_sub_q(a, w, __umul64hi(a, ws), q);  // in [0, 2q) for any a < 2^64
}
// x, y in [0, 4q) -> [0, 4q)
__device__ __forceinline__ void ct_lazy(uint64_t& x, uint64_t& y, uint64_t w, uint64_t ws,
                                        uint64_t q, uint64_t q2) {
  uint64_t u = x >= q2 ? x - q2 : x;
  const uint64_t t = shoup_lazy(y, w, ws, q);
  x = u + t;
  y = u - t + q2;
}
// x, y in [0, 2q) -> [0, 2q)
__device__ __forceinline__ void gs_lazy(uint64_t& x, uint64_t& y, uint64_t w, uint64_t ws,
                                        uint64_t q, uint64_t q2) {
  const uint64_t u = x, v = y;
  uint64_t s = u + v;
  x = s >= q2 ? s - q2 : s;
  y = shoup_lazy(u - v + q2, w, ws, q);
}
// Inverse butterfly without the reduction of x, for moduli q < 2^48: with
// every input of stage s below c = 2^s q (a multiple of q), x' = u + v < 2c
// and y' = [(u - v + c) w] in [0, 2q), so the inputs of stage s + 1 are below
// 2^(s+1) q; after the 16 stages of N = 2^16 every value is below
// 2^16 q < 2^64, and the output scaling (any 64-bit input) reduces fully.
__device__ __forceinline__ void gs_grow(uint64_t& x, uint64_t& y, uint64_t w, uint64_t ws,
                                        uint64_t q, uint64_t c) {
  const uint64_t u = x, v = y;
  x = u + v;
  y = shoup_lazy(u - v + c, w, ws, q);
}
template <bool GROW>
__device__ __forceinline__ void gs_step(uint64_t& x, uint64_t& y, uint64_t w, uint64_t ws,
                                        uint64_t q, uint64_t q2, uint64_t c) {
  if (GROW)
    gs_grow(x, y, w, ws, q, c);
  else
    gs_lazy(x, y, w, ws, q, q2);
}
template <bool GROW, bool CHAIN = true>
__device__ __forceinline__ void ct_step(uint64_t& x, uint64_t& y, uint64_t w, uint64_t ws,
                                        uint64_t q, uint64_t q2) {
  if (GROW)
    ct_grow<CHAIN>(x, y, w, ws, q, q2);
  else
    ct_lazy(x, y, w, ws, q, q2);
}
__device__ __forceinline__ uint64_t reduce4(uint64_t x, uint64_t q, uint64_t q2) {
  x = x >= q2 ? x - q2 : x;
  return x >= q ? x - q : x;
}

__device__ __forceinline__ void ct_bfly(uint64_t& x, uint64_t& y, uint64_t w, uint64_t ws,
                                        uint64_t q) {
  const uint64_t v = mul_shoup(y, w, ws, q);
  const uint64_t u = x;
  x = add_mod(u, v, q);
  y = sub_mod(u, v, q);
}
__device__ __forceinline__ void gs_bfly(uint64_t& x, uint64_t& y, uint64_t w, uint64_t ws,
                                        uint64_t q) {
  const uint64_t u = x, v = y;
  x = add_mod(u, v, q);
  y = mul_shoup(sub_mod(u, v, q), w, ws, q);
}

// ---------------------------------------------------------------- small N
template <bool INV>
__global__ void ntt_small(uint64_t* base, int log_n, const int16_t* pattern, int P,
                          const Mod* mods, const uint64_t* tw, const uint64_t* tws,
                          const uint64_t* ninv, const uint64_t* ninvs) {
  extern __shared__ uint64_t sm[];
  const size_t row = blockIdx.x;
  const int mi = pattern[row % P];
  if (mi < 0) return;
  const uint32_t N = 1u << log_n;
  const uint64_t q = mods[mi].q;
  const uint64_t* w = tw + (size_t)mi * N;
  const uint64_t* ws = tws + (size_t)mi * N;
  uint64_t* a = base + row * N;
  for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) sm[i] = a[i];
  __syncthreads();
  const uint32_t half = N >> 1;
  if (!INV) {
    for (uint32_t m = 1, lt = log_n - 1; m < N; m <<= 1, lt--) {
      for (uint32_t k = threadIdx.x; k < half; k += blockDim.x) {
        const uint32_t ib = k >> lt, j = (ib << (lt + 1)) + (k & ((1u << lt) - 1));
        ct_bfly(sm[j], sm[j + (1u << lt)], w[m + ib], ws[m + ib], q);
      }
      __syncthreads();
    }
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) a[i] = sm[i];
  } else {
    for (uint32_t m = half, lt = 0; m >= 1; m >>= 1, lt++) {
      for (uint32_t k = threadIdx.x; k < half; k += blockDim.x) {
        const uint32_t ib = k >> lt, j = (ib << (lt + 1)) + (k & ((1u << lt) - 1));
        gs_bfly(sm[j], sm[j + (1u << lt)], w[m + ib], ws[m + ib], q);
      }
      __syncthreads();
    }
    const uint64_t ni = ninv[mi], nis = ninvs[mi];
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) a[i] = mul_shoup(sm[i], ni, nis, q);
  }
}

// Shared-memory swizzle within each 16-element block: with it, every access
// pattern of the radix-8 rounds and of the chunk loads touches 16 distinct
// 8-byte banks per half-warp (without it the distance-1 round is 8-way
// conflicted).
__device__ __forceinline__ uint32_t swz(uint32_t i) {
  const uint32_t x = i >> 4;
  return i ^ ((x & 7) | ((x & 4) << 1));
}

// ---------------------------------------------------------------- radix-8 rounds
// Group g (0..511) of a chunk: elements base + k*s (k < 8), base = blk8*8s + r.
// B8 = global index of the 8s-block. Forward: distances 4s, 2s, s (stage
// indices m4 = N/(8s), 2 m4, 4 m4). Inverse: distances s, 2s, 4s.
// t8: this modulus' packed round twiddles (7 (w, w') pairs per node).
__device__ __forceinline__ uint32_t node_base(uint32_t ls, int log_n) {
  // nodes of earlier rounds (base distances 512, 64, 8 before 64, 8, 1)
  uint32_t off = 0;
  for (int r = 9; r > (int)ls; r -= 3) off += 1u << (log_n - r - 3);
  return off;
}

// The three butterfly layers of a round on the group's 8 words x.
template <bool INV, bool GROW, bool CHAIN = true>
__device__ __forceinline__ void bfly8(uint64_t* x, const ulonglong2* tt, uint32_t ls, uint64_t q,
                                      uint64_t q2) {
  if (!INV) {
#pragma unroll
    for (int k = 0; k < 4; k++) ct_step<GROW, CHAIN>(x[k], x[k + 4], tt[0].x, tt[0].y, q, q2);
    ct_step<GROW, CHAIN>(x[0], x[2], tt[1].x, tt[1].y, q, q2);
    ct_step<GROW, CHAIN>(x[1], x[3], tt[1].x, tt[1].y, q, q2);
    ct_step<GROW, CHAIN>(x[4], x[6], tt[2].x, tt[2].y, q, q2);
    ct_step<GROW, CHAIN>(x[5], x[7], tt[2].x, tt[2].y, q, q2);
#pragma unroll
    for (int k = 0; k < 4; k++) ct_step<GROW, CHAIN>(x[2 * k], x[2 * k + 1], tt[3 + k].x, tt[3 + k].y, q, q2);
  } else {
    // stages ls, ls + 1, ls + 2 of the inverse (bounds 2^s q when growing)
    const uint64_t c0 = GROW ? q << ls : 0;
#pragma unroll
    for (int k = 0; k < 4; k++)
      gs_step<GROW>(x[2 * k], x[2 * k + 1], tt[3 + k].x, tt[3 + k].y, q, q2, c0);
    gs_step<GROW>(x[0], x[2], tt[1].x, tt[1].y, q, q2, c0 << 1);
    gs_step<GROW>(x[1], x[3], tt[1].x, tt[1].y, q, q2, c0 << 1);
    gs_step<GROW>(x[4], x[6], tt[2].x, tt[2].y, q, q2, c0 << 1);
    gs_step<GROW>(x[5], x[7], tt[2].x, tt[2].y, q, q2, c0 << 1);
#pragma unroll
    for (int k = 0; k < 4; k++) gs_step<GROW>(x[k], x[k + 4], tt[0].x, tt[0].y, q, q2, c0 << 2);
  }
}

__device__ __forceinline__ void load_tw8(ulonglong2* tt, const ulonglong2* t8, uint32_t ls,
                                         uint32_t B8, int log_n) {
  const ulonglong2* T = t8 + (size_t)(node_base(ls, log_n) + B8) * 7;
#pragma unroll
  for (int k = 0; k < 7; k++) tt[k] = T[k];
}

template <bool INV, bool GROW = false, bool CHAIN = true>
__device__ __forceinline__ void round8(uint64_t* sm, uint32_t g, uint32_t ls, uint32_t chunk,
                                       int log_n, const ulonglong2* t8, uint64_t q, uint64_t q2) {
  const uint32_t blk8 = g >> ls, r = g & ((1u << ls) - 1);
  const uint32_t base = (blk8 << (ls + 3)) + r;
  uint64_t x[8];
#pragma unroll
  for (int k = 0; k < 8; k++) x[k] = sm[swz(base + ((uint32_t)k << ls))];
  ulonglong2 tt[7];
  load_tw8(tt, t8, ls, (chunk << (CHUNK_LOG - ls - 3)) + blk8, log_n);
  bfly8<INV, GROW, CHAIN>(x, tt, ls, q, q2);
#pragma unroll
  for (int k = 0; k < 8; k++) sm[swz(base + ((uint32_t)k << ls))] = x[k];
}

// The inverse's first round (distances 1, 2, 4): group g is the 8
// consecutive words 8g .. 8g+7 of the chunk, read straight from global
// memory (16-byte loads when the chunk is 16-byte aligned) instead of
// through a shared-memory copy.
template <bool GROW>
__device__ __forceinline__ void round8_inv_first(uint64_t* sm, const uint64_t* src, uint32_t g,
                                                 uint32_t chunk, int log_n, const ulonglong2* t8,
                                                 uint64_t q, uint64_t q2, bool vec) {
  const uint32_t base = g << 3;
  uint64_t x[8];
  if (vec) {
    const ulonglong2* v = reinterpret_cast<const ulonglong2*>(src + base);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const ulonglong2 p = v[k];
      x[2 * k] = p.x;
      x[2 * k + 1] = p.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = src[base + k];
  }
  ulonglong2 tt[7];
  load_tw8(tt, t8, 0, (chunk << (CHUNK_LOG - 3)) + g, log_n);
  bfly8<true, GROW>(x, tt, 0, q, q2);
#pragma unroll
  for (int k = 0; k < 8; k++) sm[swz(base + (uint32_t)k)] = x[k];
}

// Per-CTA row description produced by a descriptor's setup().
struct Row {
  int mi;            // modulus index
  uint64_t* mid;     // row used for the intermediate (and the output unless stored elsewhere)
  const uint64_t* src;   // prologue source rows
  const uint64_t* src2;  // epilogue source row
  int n_src;
  uint64_t k, ks;    // epilogue constant
  uint64_t aux;      // rescale: q of the dropped prime
  const uint64_t* src3;  // second epilogue source row (merged relinearise + rescale)
  uint64_t k2, k2s;      // its constant
  const uint8_t* ov;     // conversion overflow per coefficient (centred conversions)
  uint64_t km, kms;      // [M]_q subtracted ov times
};

constexpr int MAX_SRC = 16;

// plain forward NTT of pattern-selected rows
struct DescPlain {
  static constexpr bool CHAIN = true;  // remainder form (modarith.cuh)
  static constexpr int SLOT = NTT_SLOT_FWD;
  static constexpr bool FOLD1 = false;  // see DescModUp
  static constexpr bool COL_LOADS = false;  // see DescModDown
  uint64_t* base;
  const int16_t* pattern;
  int P;
  size_t N;
  __device__ bool setup(uint32_t blk, Row& r, uint64_t*, uint32_t, uint32_t) const {
    r.mi = pattern[blk % P];
    if (r.mi < 0) return false;
    r.mid = base + (size_t)blk * N;
    return true;
  }
  __device__ uint64_t load(const Row& r, uint32_t i, const uint64_t*, bool) const { return r.mid[i]; }
  static constexpr int EPI = 0;  // epilogue operand rows (see fwd_rows)
  __device__ void epi_load(const Row&, uint32_t, uint64_t*) const {}
  __device__ void store(const Row& r, uint32_t i, uint64_t v, uint64_t, const uint64_t*) const {
    r.mid[i] = v;
  }
};

// ModUp target row: sum_a xs[a][i] * [Dhat_a]_{m} mod m, then NTT; digit rows copy d.
struct DescModUp {
  static constexpr bool CHAIN = true;  // remainder form (modarith.cuh)
  static constexpr int SLOT = NTT_SLOT_MODUP;
  // The forward transform's first stage multiplies the upper half of the
  // row by the single twiddle w = psi^(N/2); the upper half is loaded with
  // the constants [Dhat_a w]_m instead (load_cols), so that stage is a plain
  // sum and difference (moduli below 2^50).
  static constexpr bool FOLD1 = true;
  static constexpr bool COL_LOADS = false;  // growth-tolerant rows: load_cols through FOLD1
  const uint64_t* xs;  // [B][l][N] coefficients already scaled by N^-1 Dhat^-1 (the iNTT post factor)
  const uint64_t* d;   // batch element b at d + b dstride: [l][N] NTT form
  uint64_t* ext;       // [B][beta][rows][N]
  const uint64_t* dh;  // [beta][alpha][rows]
  const uint64_t* dhs;
  size_t dstride;
  int l, beta, rows, alpha, L;
  size_t N;
  const uint64_t* dhw;  // [beta][alpha][rows]: [Dhat_a psi^(N/2)]_m
  const uint64_t* dhws;
  __device__ bool setup(uint32_t blk, Row& r, uint64_t* kc, uint32_t part, uint32_t nparts) const {
    const int rr = (int)(blk % rows);
    const int j = (int)((blk / rows) % beta);
    const size_t b = blk / ((size_t)rows * beta);
    const int lo = j * alpha, hi = min((j + 1) * alpha, l);
    uint64_t* out = ext + (((size_t)b * beta + j) * rows + rr) * N;
    if (rr >= lo && rr < hi) {
      const uint64_t* src = d + b * dstride + (size_t)rr * N;
      const size_t per = N / nparts;
      for (size_t i = part * per + threadIdx.x; i < (part + 1) * per; i += blockDim.x) out[i] = src[i];
      return false;
    }
    r.mi = rr < l ? rr : L + 1 + (rr - l);
    r.mid = out;
    r.src = xs + ((size_t)b * l + lo) * N;
    r.n_src = hi - lo;
    if (threadIdx.x < (unsigned)r.n_src) {
      const size_t ti = ((size_t)(j * alpha) + threadIdx.x) * rows + rr;
      kc[threadIdx.x] = dh[ti];
      kc[MAX_SRC + threadIdx.x] = dhs[ti];
      kc[2 * MAX_SRC + threadIdx.x] = dhw[ti];
      kc[3 * MAX_SRC + threadIdx.x] = dhws[ti];
    }
    return true;
  }
  // exact conversion sum of one element (rows with m >= 2^50; load_cols otherwise)
  __device__ uint64_t load(const Row& r, uint32_t i, const uint64_t* kc, bool) const {
    const uint64_t m = r.aux;
    uint64_t acc = 0;
    for (int a = 0; a < r.n_src; a++)
      acc = add_mod(acc, mul_shoup_t<CHAIN>(r.src[(size_t)a * N + i], kc[a], kc[MAX_SRC + a], m), m);
    return acc;
  }
  // Growth-tolerant rows (m < 2^50): the column's N1 conversion sums at once,
  // source row outermost, so a thread has N1 independent loads in flight per
  // source row (per-element sums issue one at a time and were bound by their
  // load latency); the upper half takes the constants times w = psi^(N/2)
  // (the folded first stage). Lazy three-product Shoup terms: each sum below
  // 4 n_src m.
  template <int N1>
  __device__ void load_cols(const Row& r, uint32_t c, const uint64_t* kc, uint64_t* x) const {
    const uint64_t m = r.aux;
#pragma unroll
    for (int s = 0; s < N1; s++) x[s] = 0;
    for (int a = 0; a < r.n_src; a++) {
      const uint64_t* p = r.src + (size_t)a * N + c;
      const uint64_t w0 = kc[a], w0s = kc[MAX_SRC + a];
      const uint64_t w1 = kc[2 * MAX_SRC + a], w1s = kc[3 * MAX_SRC + a];
#pragma unroll
      for (int s = 0; s < N1 / 2; s++) x[s] += shoup_approx_t<CHAIN>(p[(size_t)s * CHUNK], w0, w0s, m);
#pragma unroll
      for (int s = N1 / 2; s < N1; s++) x[s] += shoup_approx_t<CHAIN>(p[(size_t)s * CHUNK], w1, w1s, m);
    }
  }
  static constexpr int EPI = 0;  // epilogue operand rows (see fwd_rows)
  __device__ void epi_load(const Row&, uint32_t, uint64_t*) const {}
  __device__ void store(const Row& r, uint32_t i, uint64_t v, uint64_t, const uint64_t*) const {
    r.mid[i] = v;
  }
};

// Centred basis conversion of the n_src rows at r.src into modulus m = r.aux:
// sum_a y_a kc[a] - u [M]_m, with u = r.ov[i] (ModDown, merged division).
// Exact, in [0, m), one element (rows with m >= 2^50).
template <bool CHAIN>
__device__ __forceinline__ uint64_t conv_load(const Row& r, uint32_t i, const uint64_t* kc,
                                              size_t N) {
  const uint64_t m = r.aux;
  uint64_t s = 0;
  for (int a = 0; a < r.n_src; a++)
    s = add_mod(s, mul_shoup_t<CHAIN>(r.src[(size_t)a * N + i], kc[a], kc[MAX_SRC + a], m), m);
  return sub_mod(s, mul_shoup_t<CHAIN>((uint64_t)r.ov[i], r.km, r.kms, m), m);
}
// The same for the N1 elements c + s N2 of a column, for the growth-tolerant
// transforms (m < 2^50), source row outermost (N1 independent loads in flight
// per row, see DescModUp::load_cols): lazy three-product Shoup terms (each
// below 4m) plus 256 m - u [M]_m (u <= 255), values congruent to the exact
// ones and below (4 n_src + 256) m < 2^60.
template <int N1, bool CHAIN>
__device__ __forceinline__ void conv_cols(const Row& r, uint32_t c, const uint64_t* kc, size_t N,
                                          uint64_t* x) {
  const uint64_t m = r.aux;
#pragma unroll
  for (int s = 0; s < N1; s++) x[s] = 256 * m - (uint64_t)r.ov[c + (size_t)s * CHUNK] * r.km;
  for (int a = 0; a < r.n_src; a++) {
    const uint64_t* p = r.src + (size_t)a * N + c;
    const uint64_t w = kc[a], ws = kc[MAX_SRC + a];
#pragma unroll
    for (int s = 0; s < N1; s++) x[s] += shoup_approx_t<CHAIN>(p[(size_t)s * CHUNK], w, ws, m);
  }
}

// ModDown output row i of (b,k): (acc_i - NTT(sum_a y_a [Phat_a]_{q_i})) * P^-1
struct DescModDown {
  static constexpr bool CHAIN = true;  // remainder form (modarith.cuh)
  static constexpr int SLOT = NTT_SLOT_MODDOWN;
  static constexpr bool FOLD1 = false;  // see DescModUp
  // growth-tolerant rows load whole columns (conv_cols)
  static constexpr bool COL_LOADS = true;
  const uint64_t* acc;  // [BK][rows][N]; P rows already inverse-transformed and scaled
  uint64_t* out;        // [BK][l][N]
  const uint64_t* ph;   // [alpha][L+1]
  const uint64_t* phs;
  const uint64_t* pinv;  // [l]
  const uint64_t* pinvs;
  const uint8_t* ov;     // [BK][N]: u = floor(sum_a v_a / p_a + 1/2)
  const uint64_t* pq;    // [l]: P mod q_i
  const uint64_t* pqs;
  int l, rows, alpha, L;
  size_t N;
  __device__ bool setup(uint32_t blk, Row& r, uint64_t* kc, uint32_t part, uint32_t nparts) const {
    const int i = (int)(blk % l);
    const size_t bk = blk / l;
    r.mi = i;
    r.mid = out + (bk * l + i) * N;
    r.src = acc + (bk * rows + l) * N;
    r.src2 = acc + (bk * rows + i) * N;
    r.n_src = alpha;
    r.k = pinv[i];
    r.ks = pinvs[i];
    r.ov = ov + bk * N;
    r.km = pq[i];
    r.kms = pqs[i];
    if (threadIdx.x < (unsigned)alpha) {
      kc[threadIdx.x] = ph[(size_t)threadIdx.x * (L + 1) + i];
      kc[MAX_SRC + threadIdx.x] = phs[(size_t)threadIdx.x * (L + 1) + i];
    }
    return true;
  }
  __device__ uint64_t load(const Row& r, uint32_t i, const uint64_t* kc, bool grow) const {
    return conv_load<CHAIN>(r, i, kc, N);
  }
  template <int N1>
  __device__ void load_cols(const Row& r, uint32_t c, const uint64_t* kc, uint64_t* x) const {
    conv_cols<N1, CHAIN>(r, c, kc, N, x);
  }
  static constexpr int EPI = 1;
  __device__ void epi_load(const Row& r, uint32_t i, uint64_t* o) const { o[0] = r.src2[i]; }
  __device__ void store(const Row& r, uint32_t i, uint64_t v, uint64_t q, const uint64_t* o) const {
    r.mid[i] = mul_shoup(sub_mod(o[0], v, q), r.k, r.ks, q);
  }
};

// Rescale output row t of poly p: (c_t - NTT(centred(last) mod q_t)) * q_level^-1
struct DescRescale {
  static constexpr bool CHAIN = true;  // remainder form (modarith.cuh)
  static constexpr int SLOT = NTT_SLOT_RESCALE;
  static constexpr bool FOLD1 = false;  // see DescModUp
  static constexpr bool COL_LOADS = false;  // see DescModDown
  const uint64_t* in;    // [polys][level+1][N]
  const uint64_t* last;  // [polys][N] coefficient form of limb `level`
  uint64_t* out;         // [polys][level][N]
  const uint64_t* inv;   // [level]: q_level^-1 mod q_t
  const uint64_t* invs;
  uint64_t ql;
  int level;
  size_t N;
  __device__ bool setup(uint32_t blk, Row& r, uint64_t*, uint32_t, uint32_t) const {
    const int t = (int)(blk % level);
    const size_t p = blk / level;
    r.mi = t;
    r.mid = out + (p * level + t) * N;
    r.src = last + p * N;
    r.src2 = in + (p * (level + 1) + t) * N;
    r.k = inv[t];
    r.ks = invs[t];
    return true;
  }
  __device__ uint64_t load(const Row& r, uint32_t i, const uint64_t*, bool) const {
    const uint64_t x = r.src[i];
    const int64_t v = x > ql / 2 ? -(int64_t)(ql - x) : (int64_t)x;
    return smod64(v, r.aux);
  }
  static constexpr int EPI = 1;
  __device__ void epi_load(const Row& r, uint32_t i, uint64_t* o) const { o[0] = r.src2[i]; }
  __device__ void store(const Row& r, uint32_t i, uint64_t v, uint64_t q, const uint64_t* o) const {
    r.mid[i] = mul_shoup(sub_mod(o[0], v, q), r.k, r.ks, q);
  }
};

// Rescale of k c by q_level for an integer k, output row t of poly p:
//   c_t [k q_level^-1]_{q_t} - NTT(centred(last) mod q_t) [q_level^-1]_{q_t},
// with `last` the coefficient form of k c_level (the inverse transform's post
// factor carries k) and c read in place (poly p at in + p in_stride).
struct DescRescaleScaled {
  static constexpr bool CHAIN = true;  // remainder form (modarith.cuh)
  static constexpr int SLOT = NTT_SLOT_RESCALE;
  static constexpr bool FOLD1 = false;  // see DescModUp
  static constexpr bool COL_LOADS = false;  // see DescModDown
  const uint64_t* in;
  size_t in_stride;
  const uint64_t* last;   // [polys][N]
  uint64_t* out;          // [polys][level][N]
  const uint64_t* inv;    // [level]: q_level^-1 mod q_t
  const uint64_t* invs;
  const uint64_t* kinv;   // [level]: k q_level^-1 mod q_t
  const uint64_t* kinvs;
  uint64_t ql;
  int level;
  size_t N;
  __device__ bool setup(uint32_t blk, Row& r, uint64_t*, uint32_t, uint32_t) const {
    const int t = (int)(blk % level);
    const size_t p = blk / level;
    r.mi = t;
    r.mid = out + (p * level + t) * N;
    r.src = last + p * N;
    r.src2 = in + p * in_stride + (size_t)t * N;
    r.k = inv[t];
    r.ks = invs[t];
    r.k2 = kinv[t];
    r.k2s = kinvs[t];
    return true;
  }
  __device__ uint64_t load(const Row& r, uint32_t i, const uint64_t*, bool) const {
    const uint64_t x = r.src[i];
    const int64_t v = x > ql / 2 ? -(int64_t)(ql - x) : (int64_t)x;
    return smod64(v, r.aux);
  }
  static constexpr int EPI = 1;
  __device__ void epi_load(const Row& r, uint32_t i, uint64_t* o) const { o[0] = r.src2[i]; }
  __device__ void store(const Row& r, uint32_t i, uint64_t v, uint64_t q, const uint64_t* o) const {
    r.mid[i] = sub_mod(mul_shoup(o[0], r.k2, r.k2s, q), mul_shoup(v, r.k, r.ks, q), q);
  }
};

// Column and chunk phases of the forward cluster NTT (see ntt_fwd_cl).
template <int N1, class D, bool GROW>
__device__ __forceinline__ void fwd_rows(const D& d, Row& r, int log_n, const ulonglong2* t8,
                                         uint64_t q, const uint64_t* kc, const ulonglong2* ctw,
                                         uint64_t* sm) {
  constexpr int CS = fwd_cs<N1>();
  constexpr int CPC = N1 / CS;
  const uint64_t q2 = 2 * q;
  const uint64_t w1s = GROW ? ~0ull / q : 0;  // floor(2^64 / q) for odd q
  const uint32_t rank = CS > 1 ? (uint32_t)cg::this_cluster().block_rank() : 0;
  const uint32_t g = threadIdx.x;
  uint32_t own[CS];  // cluster-window address of each CTA's chunks
#pragma unroll
  for (int k = 0; k < CS; k++) own[k] = CS > 1 ? dsmem_addr(sm, k) : 0;
  constexpr uint32_t COLS = CHUNK / CS;
  for (uint32_t c = rank * COLS + g; c < (rank + 1) * COLS; c += ROW_THREADS) {
    uint64_t x[N1];
    int m0 = 1;  // first column stage still to run
    if constexpr (D::FOLD1 && GROW) {
      // first stage folded into the loads: the upper half's t = w y comes
      // with the loads, and u - t + cw with cw = 4 n_src q (a multiple of q
      // above t) stays >= 0
      const uint64_t cw = 4 * (uint64_t)r.n_src * q;
      d.template load_cols<N1>(r, c, kc, x);
#pragma unroll
      for (int s = 0; s < N1 / 2; s++) {
        const uint64_t u = x[s], t = x[s + N1 / 2];
        x[s] = u + t;
        x[s + N1 / 2] = u - t + cw;
      }
      m0 = 2;
    } else if constexpr (D::COL_LOADS && GROW) {
      d.template load_cols<N1>(r, c, kc, x);
    } else {
#pragma unroll
      for (int s = 0; s < N1; s++) x[s] = d.load(r, c + (uint32_t)s * CHUNK, kc, GROW);
    }
#pragma unroll
    for (int m = 1; m < N1; m <<= 1) {
      if (m < m0) continue;
      const int t1 = N1 / (2 * m);
#pragma unroll
      for (int i = 0; i < m; i++) {
        const ulonglong2 tv = ctw[m + i];
#pragma unroll
        for (int jj = 0; jj < t1; jj++)
          ct_step<GROW, D::CHAIN>(x[i * 2 * t1 + jj], x[i * 2 * t1 + jj + t1], tv.x, tv.y, q, q2);
      }
    }
#pragma unroll
    for (int s = 0; s < N1; s++) {
      const uint32_t e = (s % CPC) * CHUNK + swz(c);
      if constexpr (CS > 1)
        st_dsmem(own[s / CPC] + e * 8, x[s]);
      else
        sm[e] = x[s];
    }
  }
  if constexpr (CS > 1)
    cg::this_cluster().sync();
  else
    __syncthreads();
  // chunks in pairs (CPC is even): one group of each chunk per thread
  for (int lc = 0; lc < CPC; lc += 2) {
    const uint32_t chunk = rank * CPC + lc;
    uint64_t* s = sm + lc * CHUNK;
#pragma unroll
    for (int ls = 9; ls >= 0; ls -= 3) {
      round8<false, GROW, D::CHAIN>(s, g, ls, chunk, log_n, t8, q, q2);
      round8<false, GROW, D::CHAIN>(s + CHUNK, g, ls, chunk + 1, log_n, t8, q, q2);
      __syncthreads();
    }
    // stored through shared memory so that a warp writes 256 contiguous
    // bytes per instruction (the last round's groups are 8 consecutive
    // words per thread, which would make every store instruction strided).
    // The epilogue's global operands (D::EPI rows) are loaded for a group of
    // G elements before any of them is stored: a load cannot be moved above
    // a store the compiler cannot tell apart from it, so element by element
    // a thread would have one load in flight.
    constexpr int SPT = 2 * CHUNK / ROW_THREADS;
    constexpr int G = D::EPI > 1 ? 4 : 8;
    constexpr int NE = D::EPI > 0 ? D::EPI : 1;
#pragma unroll
    for (int k0 = 0; k0 < SPT; k0 += G) {
      uint64_t o[G][NE];
#pragma unroll
      for (int k = 0; k < G; k++)
        d.epi_load(r, chunk * CHUNK + g + (uint32_t)(k0 + k) * ROW_THREADS, o[k]);
#pragma unroll
      for (int k = 0; k < G; k++) {
        const uint32_t i = g + (uint32_t)(k0 + k) * ROW_THREADS;
        const uint64_t v = s[(i & ~(CHUNK - 1)) + swz(i & (CHUNK - 1))];
        d.store(r, chunk * CHUNK + i, GROW ? reduce_full(v, q, w1s) : reduce4(v, q, q2), q, o[k]);
      }
    }
  }
}

// HMult's relinearise + rescale, output row i < level of (b, k):
//   d_k[i] q_level^-1 + (acc_k[i] - NTT(sum_m y_m [M/m]_{q_i})) M^-1,
// y_m the D rows of acc (level .. level+alpha) already inverse-transformed and
// scaled by (M/m)^-1, with y_level = P d_k + acc_k on q_level.
struct DescRelinRescale {
  static constexpr bool CHAIN = false;  // remainder form (modarith.cuh)
  static constexpr int SLOT = NTT_SLOT_RELIN_RESCALE;
  static constexpr bool FOLD1 = false;  // see DescModUp
  static constexpr bool COL_LOADS = true;
  const uint64_t* acc;    // [BK][rows][N]
  const uint64_t* d;      // [B][3][level+1][N] tensor product
  uint64_t* out;          // [BK][level][N]
  const uint64_t* mh;     // [alpha+1][level+1]: (M/m) mod q_i
  const uint64_t* mhs;
  const uint64_t* minv;   // [level+1]: M^-1 mod q_i
  const uint64_t* minvs;
  const uint64_t* qlinv;  // [L+1]: q_level^-1 mod q_t
  const uint64_t* qlinvs;
  const uint8_t* ov;      // [BK][N]: u = floor(sum_m v_m / m + 1/2)
  const uint64_t* mq;     // [level+1]: M mod q_i
  const uint64_t* mqs;
  int level, rows, alpha;
  size_t N;
  __device__ bool setup(uint32_t blk, Row& r, uint64_t* kc, uint32_t, uint32_t) const {
    const int i = (int)(blk % level);
    const size_t bk = blk / level;
    const size_t b = bk / 2, k = bk % 2;
    const int l = level + 1;
    r.mi = i;
    r.mid = out + (bk * level + i) * N;
    r.src = acc + (bk * rows + level) * N;
    r.n_src = alpha + 1;
    r.src2 = acc + (bk * rows + i) * N;
    r.src3 = d ? d + ((b * 3 + k) * l + i) * N : nullptr;  // null: no tensor term
    r.k = minv[i];
    r.ks = minvs[i];
    r.k2 = qlinv[i];
    r.k2s = qlinvs[i];
    r.ov = ov + bk * N;
    r.km = mq[i];
    r.kms = mqs[i];
    if (threadIdx.x < (unsigned)(alpha + 1)) {
      kc[threadIdx.x] = mh[(size_t)threadIdx.x * l + i];
      kc[MAX_SRC + threadIdx.x] = mhs[(size_t)threadIdx.x * l + i];
    }
    return true;
  }
  __device__ uint64_t load(const Row& r, uint32_t i, const uint64_t* kc, bool grow) const {
    return conv_load<CHAIN>(r, i, kc, N);
  }
  template <int N1>
  __device__ void load_cols(const Row& r, uint32_t c, const uint64_t* kc, uint64_t* x) const {
    conv_cols<N1, CHAIN>(r, c, kc, N, x);
  }
  static constexpr int EPI = 2;
  __device__ void epi_load(const Row& r, uint32_t i, uint64_t* o) const {
    o[0] = r.src2[i];
    o[1] = r.src3 ? r.src3[i] : 0;
  }
  __device__ void store(const Row& r, uint32_t i, uint64_t v, uint64_t q, const uint64_t* o) const {
    const uint64_t y = mul_shoup_t<CHAIN>(sub_mod(o[0], v, q), r.k, r.ks, q);
    r.mid[i] = r.src3 ? add_mod(mul_shoup_t<CHAIN>(o[1], r.k2, r.k2s, q), y, q) : y;
  }
};

// Forward NTT of one row per cluster of CS = fwd_cs<N1>() CTAs, two chunks per CTA.
// CTA `rank` owns chunks [rank*CPC, (rank+1)*CPC) of the row in shared memory.
// Column phase: the CTA transforms columns [rank*CHUNK/CS, ...) from the
// prologue loads and writes element s of each column into the shared memory
// of the CTA owning chunk s (distributed shared memory). After a cluster
// barrier each CTA runs the radix-8 rounds on its own chunks in place and
// writes the results through the epilogue. The row never round-trips
// through global memory.
template <int N1, class D, int MINB = CTAS_PER_SM>
__global__ void __launch_bounds__(ROW_THREADS, MINB)
    ntt_fwd_cl(D d, int log_n, const Mod* mods, const uint64_t* tw, const uint64_t* tws,
               const ulonglong2* tw8, size_t nodes) {
  constexpr int CS = fwd_cs<N1>();
  extern __shared__ uint64_t sm[];  // CPC = N1 / CS chunks
  __shared__ uint64_t kc[4 * MAX_SRC];
  __shared__ ulonglong2 ctw[N1];  // column-stage twiddles (nodes 1 .. N1-1)
  const uint32_t rank = CS > 1 ? (uint32_t)cg::this_cluster().block_rank() : 0;
  const uint32_t row = blockIdx.x / CS;
  Row r;
  r.n_src = 0;
  if (!d.setup(row, r, kc, rank, CS)) return;  // same decision on every CTA of the cluster
  const size_t N = (size_t)N1 * CHUNK;
  const uint64_t q = mods[r.mi].q;
  r.aux = q;
  const ulonglong2* t8 = tw8 + (size_t)r.mi * nodes * 7;
  const uint32_t g = threadIdx.x;
  if (g < (uint32_t)N1) ctw[g] = make_ulonglong2(tw[(size_t)r.mi * N + g], tws[(size_t)r.mi * N + g]);
  __syncthreads();
  // every CTA of a cluster works on the same row, so the branch is uniform
  if (q < (1ull << 50))
    fwd_rows<N1, D, true>(d, r, log_n, t8, q, kc, ctw, sm);
  else
    fwd_rows<N1, D, false>(d, r, log_n, t8, q, kc, ctw, sm);
}

// Both phases of the inverse transform of one row (see ntt_inv_cl).
template <int N1, bool GROW>
__device__ __forceinline__ void inv_rows(uint64_t* a, const uint64_t* as, uint64_t* sm,
                                         const ulonglong2* ctw, const ulonglong2* t8, int log_n,
                                         uint64_t q, uint64_t pv, uint64_t pvs, uint32_t rank) {
  constexpr int CS = inv_cs<N1>();
  constexpr int CPC = N1 / CS;
  const uint64_t q2 = 2 * q;
  const uint32_t g = threadIdx.x;
  // chunks in pairs (CPC is even): one group of each chunk per thread
  for (int lc = 0; lc < CPC; lc += 2) {
    const uint32_t chunk = rank * CPC + lc;
    uint64_t* s = sm + lc * CHUNK;
    const uint64_t* ac = as + (size_t)chunk * CHUNK;
    const bool vec = (reinterpret_cast<uintptr_t>(ac) & 15) == 0;
    round8_inv_first<GROW>(s, ac, g, chunk, log_n, t8, q, q2, vec);
    round8_inv_first<GROW>(s + CHUNK, ac + CHUNK, g, chunk + 1, log_n, t8, q, q2, vec);
    __syncthreads();
#pragma unroll
    for (int ls = 3; ls <= 9; ls += 3) {
      round8<true, GROW>(s, g, ls, chunk, log_n, t8, q, q2);
      round8<true, GROW>(s + CHUNK, g, ls, chunk + 1, log_n, t8, q, q2);
      __syncthreads();
    }
  }
  uint32_t own[CS];  // cluster-window address of each CTA's chunks
  if constexpr (CS > 1) cg::this_cluster().sync();
#pragma unroll
  for (int k = 0; k < CS; k++) own[k] = CS > 1 ? dsmem_addr(sm, k) : 0;
  constexpr uint32_t COLS = CHUNK / CS;
  for (uint32_t c = rank * COLS + g; c < (rank + 1) * COLS; c += ROW_THREADS) {
    uint64_t x[N1];
#pragma unroll
    for (int s = 0; s < N1; s++) {
      const uint32_t e = (s % CPC) * CHUNK + swz(c);
      if constexpr (CS > 1)
        x[s] = ld_dsmem(own[s / CPC] + e * 8);
      else
        x[s] = sm[e];
    }
#pragma unroll
    for (int m = N1 / 2; m >= 1; m >>= 1) {
      const int t1 = N1 / (2 * m);
      const uint64_t cs = GROW ? (q << CHUNK_LOG) * (uint64_t)t1 : 0;  // stage 12 + log2 t1
#pragma unroll
      for (int i = 0; i < m; i++) {
        const ulonglong2 tv = ctw[m + i];
#pragma unroll
        for (int jj = 0; jj < t1; jj++)
          gs_step<GROW>(x[i * 2 * t1 + jj], x[i * 2 * t1 + jj + t1], tv.x, tv.y, q, q2, cs);
      }
    }
#pragma unroll
    for (int s = 0; s < N1; s++) a[c + (size_t)s * CHUNK] = mul_shoup(x[s], pv, pvs, q);
  }
  if constexpr (CS > 1) cg::this_cluster().sync();  // peers may still read this CTA's chunks
}

// Inverse NTT of pattern-selected rows, one row per cluster: each CTA loads
// and transforms its own chunks, then (after a cluster barrier) transforms
// its share of the columns, reading the elements from the owners' shared
// memory, and writes the row scaled by post[row % P] (default N^-1).
template <int N1, int MINB = CTAS_PER_SM>
__global__ void __launch_bounds__(ROW_THREADS, MINB)
    ntt_inv_cl(uint64_t* base, const uint64_t* src, size_t src_stride, int log_n,
               const int16_t* pattern, int P, const Mod* mods,
               const uint64_t* tw, const uint64_t* tws, const uint64_t* ninv,
               const uint64_t* ninvs, const uint64_t* post, const uint64_t* posts,
               const ulonglong2* tw8, size_t nodes) {
  constexpr int CS = inv_cs<N1>();
  extern __shared__ uint64_t sm[];
  __shared__ ulonglong2 ctw[N1];  // column-stage twiddles (nodes 1 .. N1-1)
  const uint32_t rank = CS > 1 ? (uint32_t)cg::this_cluster().block_rank() : 0;
  const size_t row = blockIdx.x / CS;
  const int mi = pattern[row % P];
  if (mi < 0) return;  // same decision on every CTA of the cluster
  const size_t N = (size_t)N1 * CHUNK;
  const uint64_t q = mods[mi].q;
  const ulonglong2* t8 = tw8 + (size_t)mi * nodes * 7;
  uint64_t* a = base + row * N;
  // source rows: in place, or row i of period p at src + p src_stride + i N
  const uint64_t* as = src ? src + (row / P) * src_stride + (row % P) * N : a;
  const uint64_t pv = post ? post[row % P] : ninv[mi];
  const uint64_t pvs = post ? posts[row % P] : ninvs[mi];
  const uint32_t g = threadIdx.x;
  if (g < (uint32_t)N1) ctw[g] = make_ulonglong2(tw[(size_t)mi * N + g], tws[(size_t)mi * N + g]);
  // every CTA of a cluster works on the same row, so the branch is uniform
  if (q < (1ull << 48))
    inv_rows<N1, true>(a, as, sm, ctw, t8, log_n, q, pv, pvs, rank);
  else
    inv_rows<N1, false>(a, as, sm, ctw, t8, log_n, q, pv, pvs, rank);
}

template <int N1, int CS, int MINB, class K, class... Args>
void launch_cl(Ctx& c, K kernel, size_t n_rows, Args... args) {
  constexpr int CPC = N1 / CS;
  const size_t smem = (size_t)CPC * CHUNK * 8;
  static bool attr[64] = {};
  if (!attr[c.device & 63]) {
    CK_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (CS > 1) CK_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 0));
    attr[c.device & 63] = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n_rows * CS));
  cfg.blockDim = dim3(ROW_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c.stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  CK_CUDA(cudaLaunchKernelEx(&cfg, kernel, args...));
}

template <class D>
void launch_fwd(Ctx& c, size_t n_rows, const D& d) {
  if (n_rows == 0) return;
  const uint64_t* tw = c.d_tw.u64();
  const uint64_t* tws = c.d_tws.u64();
  const ulonglong2* t8 = static_cast<const ulonglong2*>(c.d_tw8.p);
  const size_t nd = c.tw8_nodes;
  const int ln = c.log_n;
  const Mod* md = c.dmod();
  const bool one = c.ntt_minb[D::SLOT] == 1;
  switch (c.log_n - CHUNK_LOG) {
    case 1: launch_cl<2, fwd_cs<2>(), 2>(c, ntt_fwd_cl<2, D>, n_rows, d, ln, md, tw, tws, t8, nd); break;
    case 2: launch_cl<4, fwd_cs<4>(), 2>(c, ntt_fwd_cl<4, D>, n_rows, d, ln, md, tw, tws, t8, nd); break;
    case 3:
      if (one) launch_cl<8, fwd_cs<8>(), 1>(c, ntt_fwd_cl<8, D, 1>, n_rows, d, ln, md, tw, tws, t8, nd);
      else launch_cl<8, fwd_cs<8>(), 2>(c, ntt_fwd_cl<8, D>, n_rows, d, ln, md, tw, tws, t8, nd);
      break;
    case 4:
      if (one) launch_cl<16, fwd_cs<16>(), 1>(c, ntt_fwd_cl<16, D, 1>, n_rows, d, ln, md, tw, tws, t8, nd);
      else launch_cl<16, fwd_cs<16>(), 2>(c, ntt_fwd_cl<16, D>, n_rows, d, ln, md, tw, tws, t8, nd);
      break;
    default: throw Error(CKKS_ERR_UNSUPPORTED, "NTT size");
  }
}

void launch_inv(Ctx& c, size_t n_rows, uint64_t* base, const int16_t* pattern, int P,
                const uint64_t* post, const uint64_t* posts, const uint64_t* src = nullptr,
                size_t src_stride = 0) {
  if (n_rows == 0) return;
  const uint64_t* tw = c.d_itw.u64();
  const uint64_t* tws = c.d_itws.u64();
  const uint64_t* ni = c.d_ninv.u64();
  const uint64_t* nis = c.d_ninvs.u64();
  const ulonglong2* t8 = static_cast<const ulonglong2*>(c.d_itw8.p);
  const size_t nd = c.tw8_nodes;
  const int ln = c.log_n;
  const Mod* md = c.dmod();
  const bool one = c.ntt_minb[NTT_SLOT_INV] == 1;
  switch (c.log_n - CHUNK_LOG) {
    case 1: launch_cl<2, inv_cs<2>(), 2>(c, ntt_inv_cl<2>, n_rows, base, src, src_stride, ln, pattern, P, md, tw, tws, ni, nis, post, posts, t8, nd); break;
    case 2: launch_cl<4, inv_cs<4>(), 2>(c, ntt_inv_cl<4>, n_rows, base, src, src_stride, ln, pattern, P, md, tw, tws, ni, nis, post, posts, t8, nd); break;
    case 3:
      if (one) launch_cl<8, inv_cs<8>(), 1>(c, ntt_inv_cl<8, 1>, n_rows, base, src, src_stride, ln, pattern, P, md, tw, tws, ni, nis, post, posts, t8, nd);
      else launch_cl<8, inv_cs<8>(), 2>(c, ntt_inv_cl<8>, n_rows, base, src, src_stride, ln, pattern, P, md, tw, tws, ni, nis, post, posts, t8, nd);
      break;
    case 4:
      if (one) launch_cl<16, inv_cs<16>(), 1>(c, ntt_inv_cl<16, 1>, n_rows, base, src, src_stride, ln, pattern, P, md, tw, tws, ni, nis, post, posts, t8, nd);
      else launch_cl<16, inv_cs<16>(), 2>(c, ntt_inv_cl<16>, n_rows, base, src, src_stride, ln, pattern, P, md, tw, tws, ni, nis, post, posts, t8, nd);
      break;
    default: throw Error(CKKS_ERR_UNSUPPORTED, "NTT size");
  }
}

template <bool INV>
void ntt_run(Ctx& c, uint64_t* base, size_t n_rows, const int16_t* pattern, int P, size_t active) {
  if (n_rows == 0) return;
  const double bytes = 2.0 * (double)std::min(active, n_rows) * (double)c.N * 8.0;
  const double bf = (double)std::min(active, n_rows) * (double)(c.N / 2) * c.log_n;  // butterflies
  if (c.log_n <= CHUNK_LOG) {
    const int threads = std::min<int>(256, (int)(c.N / 2));
    Launch L_(c, K_NTT_SMALL, bytes, bf);
    ntt_small<INV><<<(unsigned)n_rows, threads, c.N * 8, c.stream>>>(
        base, c.log_n, pattern, P, c.dmod(),
        static_cast<const uint64_t*>(INV ? c.d_itw.p : c.d_tw.p),
        static_cast<const uint64_t*>(INV ? c.d_itws.p : c.d_tws.p), c.d_ninv.u64(), c.d_ninvs.u64());
    CK_CUDA(cudaGetLastError());
  } else if (!INV) {
    Launch L_(c, K_NTT_FWD, bytes, bf);
    launch_fwd(c, n_rows, DescPlain{base, pattern, P, c.N});
  } else {
    Launch L_(c, K_NTT_INV, bytes, bf + (double)std::min(active, n_rows) * c.N);
    launch_inv(c, n_rows, base, pattern, P, nullptr, nullptr);
  }
}

}  // namespace

void ntt_forward(Ctx& c, uint64_t* base, size_t n_rows, const int16_t* pattern, int P,
                 size_t active) {
  ntt_run<false>(c, base, n_rows, pattern, P, active);
}
void ntt_inverse(Ctx& c, uint64_t* base, size_t n_rows, const int16_t* pattern, int P,
                 size_t active) {
  ntt_run<true>(c, base, n_rows, pattern, P, active);
}

bool ntt_fused_available(const Ctx& c) {
  return c.fused && c.log_n > CHUNK_LOG && c.log_n <= CHUNK_LOG + 4;
}

void ntt_inverse_post(Ctx& c, uint64_t* base, size_t n_rows, const int16_t* pattern, int P,
                      const uint64_t* post, const uint64_t* posts, size_t active,
                      const uint64_t* src, size_t src_stride) {
  const double rws = (double)std::min(active, n_rows);
  Launch L_(c, K_NTT_INV, 2.0 * rws * (double)c.N * 8.0, rws * ((double)(c.N / 2) * c.log_n + c.N));
  launch_inv(c, n_rows, base, pattern, P, post, posts, src, src_stride);
}

void ntt_modup_fused(Ctx& c, const uint64_t* xs, const uint64_t* d, size_t d_stride, size_t B,
                     int level, uint64_t* ext) {
  ConvTables& T = c.tables(level);
  if (c.alpha > MAX_SRC) throw Error(CKKS_ERR_UNSUPPORTED, "alpha > 16");
  const double W8 = (double)c.N * 8.0;
  // reads: alpha scaled source rows per target row (L2-resident per digit) and
  // the digit rows once; writes every extended row once
  const double out_rows = (double)B * ((double)T.beta * T.rows - T.l);
  Launch L_(c, K_MODUP_NTT, W8 * (double)B * (2.0 * T.l + (double)T.beta * T.rows),
            out_rows * ((double)(c.N / 2) * c.log_n + (double)c.alpha * c.N));
  DescModUp dsc{xs, d, ext, T.dh.u64(), T.dh_s.u64(), d_stride, T.l, T.beta, T.rows, c.alpha, c.L,
                c.N, T.dhw.u64(), T.dhw_s.u64()};
  launch_fwd(c, B * T.beta * T.rows, dsc);
}

void ntt_moddown_fused(Ctx& c, const uint64_t* acc, const uint8_t* ov, size_t BK, int level,
                       uint64_t* out) {
  ConvTables& T = c.tables(level);
  const double W8 = (double)c.N * 8.0;
  Launch L_(c, K_MODDOWN_NTT, W8 * (double)BK * (c.alpha + 2.0 * T.l),
            (double)BK * T.l * ((double)(c.N / 2) * c.log_n + (c.alpha + 1.0) * c.N));
  DescModDown dsc{acc, out, c.d_md_ph.u64(), c.d_md_ph_s.u64(), T.md_pinv.u64(), T.md_pinv_s.u64(),
                  ov, T.md_pq.u64(), T.md_pq_s.u64(), T.l, T.rows, c.alpha, c.L, c.N};
  launch_fwd(c, BK * T.l, dsc);
}

void ntt_relin_rescale_fused(Ctx& c, const uint64_t* acc, const uint64_t* d, const uint8_t* ov,
                             size_t B, int level, uint64_t* out) {
  ConvTables& T = c.tables(level);
  if (c.alpha + 1 > MAX_SRC) throw Error(CKKS_ERR_UNSUPPORTED, "alpha > 15");
  const double W8 = (double)c.N * 8.0;
  const double BK = 2.0 * (double)B;
  Launch L_(c, K_RR_NTT, W8 * BK * (c.alpha + 1.0 + (d ? 3.0 : 2.0) * level),
            BK * level * ((double)(c.N / 2) * c.log_n + (c.alpha + 3.0) * c.N));
  DescRelinRescale dsc{acc, d, out, T.rr_mh.u64(), T.rr_mh_s.u64(), T.rr_minv.u64(),
                       T.rr_minv_s.u64(), c.d_rs_inv.u64() + (size_t)level * (c.L + 1),
                       c.d_rs_invs.u64() + (size_t)level * (c.L + 1), ov, T.rr_mq.u64(),
                       T.rr_mq_s.u64(), level, T.rows, c.alpha, c.N};
  launch_fwd(c, 2 * B * level, dsc);
}

void ntt_rescale_fused(Ctx& c, const uint64_t* in, const uint64_t* last, size_t polys, int level,
                       uint64_t* out) {
  const double W8 = (double)c.N * 8.0;
  Launch L_(c, K_RESCALE_NTT, W8 * (double)polys * (1.0 + 2.0 * level),
            (double)polys * level * ((double)(c.N / 2) * c.log_n + c.N));
  DescRescale dsc{in, last, out, c.d_rs_inv.u64() + (size_t)level * (c.L + 1),
                  c.d_rs_invs.u64() + (size_t)level * (c.L + 1), c.mod[level], level, c.N};
  launch_fwd(c, polys * level, dsc);
}

void ntt_rescale_scaled_fused(Ctx& c, const uint64_t* in, size_t in_stride, const uint64_t* last,
                              size_t polys, int level, const uint64_t* kinv, const uint64_t* kinvs,
                              uint64_t* out) {
  const double W8 = (double)c.N * 8.0;
  Launch L_(c, K_RESCALE_NTT, W8 * (double)polys * (1.0 + 2.0 * level),
            (double)polys * level * ((double)(c.N / 2) * c.log_n + 2.0 * c.N));
  DescRescaleScaled dsc{in, in_stride, last, out, c.d_rs_inv.u64() + (size_t)level * (c.L + 1),
                        c.d_rs_invs.u64() + (size_t)level * (c.L + 1), kinv, kinvs, c.mod[level],
                        level, c.N};
  launch_fwd(c, polys * level, dsc);
}

}  // namespace ck
