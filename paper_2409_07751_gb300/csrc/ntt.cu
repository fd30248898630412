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

#include "modarith.cuh"

namespace ck {

namespace {

constexpr int CHUNK_LOG = 12;
constexpr int CHUNK = 1 << CHUNK_LOG;  // N2
constexpr int ROW_THREADS = 512;       // one radix-8 group per thread per round

__device__ __forceinline__ uint64_t shoup_lazy(uint64_t a, uint64_t w, uint64_t ws, uint64_t q) {
  return a * w - __umul64hi(a, ws) * q;  // in [0, 2q) for any a < 2^64
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

// ---------------------------------------------------------------- radix-8 rounds
// Group g (0..511) of a chunk: elements base + k*s (k < 8), base = blk8*8s + r.
// B8 = global index of the 8s-block. Forward: distances 4s, 2s, s (stage
// indices m4 = N/(8s), 2 m4, 4 m4). Inverse: distances s, 2s, 4s.
template <bool INV>
__device__ __forceinline__ void round8(uint64_t* sm, uint32_t g, uint32_t ls, uint32_t chunk,
                                       int log_n, const uint64_t* w, const uint64_t* ws,
                                       uint64_t q, uint64_t q2) {
  const uint32_t blk8 = g >> ls, r = g & ((1u << ls) - 1);
  const uint32_t base = (blk8 << (ls + 3)) + r;
  const uint32_t B8 = (chunk << (CHUNK_LOG - ls - 3)) + blk8;
  const uint32_t m4 = 1u << (log_n - ls - 3);
  uint64_t x[8];
#pragma unroll
  for (int k = 0; k < 8; k++) x[k] = sm[base + ((uint32_t)k << ls)];
  if (!INV) {
    {
      const uint32_t i = m4 + B8;
      const uint64_t a = w[i], as = ws[i];
#pragma unroll
      for (int k = 0; k < 4; k++) ct_lazy(x[k], x[k + 4], a, as, q, q2);
    }
    {
      const uint32_t i = 2 * m4 + 2 * B8;
      const uint64_t a = w[i], as = ws[i], b = w[i + 1], bs = ws[i + 1];
      ct_lazy(x[0], x[2], a, as, q, q2);
      ct_lazy(x[1], x[3], a, as, q, q2);
      ct_lazy(x[4], x[6], b, bs, q, q2);
      ct_lazy(x[5], x[7], b, bs, q, q2);
    }
    {
      const uint32_t i = 4 * m4 + 4 * B8;
#pragma unroll
      for (int k = 0; k < 4; k++) ct_lazy(x[2 * k], x[2 * k + 1], w[i + k], ws[i + k], q, q2);
    }
  } else {
    {
      const uint32_t i = 4 * m4 + 4 * B8;
#pragma unroll
      for (int k = 0; k < 4; k++) gs_lazy(x[2 * k], x[2 * k + 1], w[i + k], ws[i + k], q, q2);
    }
    {
      const uint32_t i = 2 * m4 + 2 * B8;
      const uint64_t a = w[i], as = ws[i], b = w[i + 1], bs = ws[i + 1];
      gs_lazy(x[0], x[2], a, as, q, q2);
      gs_lazy(x[1], x[3], a, as, q, q2);
      gs_lazy(x[4], x[6], b, bs, q, q2);
      gs_lazy(x[5], x[7], b, bs, q, q2);
    }
    {
      const uint32_t i = m4 + B8;
      const uint64_t a = w[i], as = ws[i];
#pragma unroll
      for (int k = 0; k < 4; k++) gs_lazy(x[k], x[k + 4], a, as, q, q2);
    }
  }
#pragma unroll
  for (int k = 0; k < 8; k++) sm[base + ((uint32_t)k << ls)] = x[k];
}

// column transform of N1 elements (stride CHUNK) in registers
template <int N1, bool INV>
__device__ __forceinline__ void column(uint64_t* a, const uint64_t* w, const uint64_t* ws,
                                       uint64_t q, uint64_t q2, uint64_t ni, uint64_t nis) {
  uint64_t x[N1];
#pragma unroll
  for (int s = 0; s < N1; s++) x[s] = a[(size_t)s * CHUNK];
  if (!INV) {
#pragma unroll
    for (int m = 1; m < N1; m <<= 1) {
      const int t1 = N1 / (2 * m);
#pragma unroll
      for (int i = 0; i < m; i++) {
        const uint64_t wv = w[m + i], wsv = ws[m + i];
#pragma unroll
        for (int jj = 0; jj < t1; jj++) ct_lazy(x[i * 2 * t1 + jj], x[i * 2 * t1 + jj + t1], wv, wsv, q, q2);
      }
    }
#pragma unroll
    for (int s = 0; s < N1; s++) a[(size_t)s * CHUNK] = x[s];
  } else {
#pragma unroll
    for (int m = N1 / 2; m >= 1; m >>= 1) {
      const int t1 = N1 / (2 * m);
#pragma unroll
      for (int i = 0; i < m; i++) {
        const uint64_t wv = w[m + i], wsv = ws[m + i];
#pragma unroll
        for (int jj = 0; jj < t1; jj++) gs_lazy(x[i * 2 * t1 + jj], x[i * 2 * t1 + jj + t1], wv, wsv, q, q2);
      }
    }
#pragma unroll
    for (int s = 0; s < N1; s++) a[(size_t)s * CHUNK] = mul_shoup(x[s], ni, nis, q);
  }
}

// One CTA per row: forward = columns then chunks; inverse = chunks then columns.
template <int N1, bool INV>
__global__ void __launch_bounds__(ROW_THREADS, 1)
    ntt_row(uint64_t* base, int log_n, const int16_t* pattern, int P, const Mod* mods,
            const uint64_t* tw, const uint64_t* tws, const uint64_t* ninv, const uint64_t* ninvs) {
  __shared__ uint64_t s[CHUNK];
  const size_t row = blockIdx.x;
  const int mi = pattern[row % P];
  if (mi < 0) return;
  const size_t N = (size_t)N1 * CHUNK;
  const uint64_t q = mods[mi].q, q2 = 2 * q;
  const uint64_t* w = tw + (size_t)mi * N;
  const uint64_t* ws = tws + (size_t)mi * N;
  uint64_t* a = base + row * N;
  const uint64_t ni = ninv[mi], nis = ninvs[mi];
  const uint32_t g = threadIdx.x;
  if (!INV) {
    for (uint32_t c = g; c < CHUNK; c += ROW_THREADS) column<N1, false>(a + c, w, ws, q, q2, ni, nis);
    __syncthreads();
  }
  for (uint32_t chunk = 0; chunk < (uint32_t)N1; chunk++) {
    uint64_t* ac = a + (size_t)chunk * CHUNK;
    for (uint32_t i = g; i < CHUNK; i += ROW_THREADS) s[i] = ac[i];
    __syncthreads();
    if (!INV) {
#pragma unroll
      for (int ls = 9; ls >= 0; ls -= 3) {
        round8<false>(s, g, ls, chunk, log_n, w, ws, q, q2);
        __syncthreads();
      }
      for (uint32_t i = g; i < CHUNK; i += ROW_THREADS) ac[i] = reduce4(s[i], q, q2);
    } else {
#pragma unroll
      for (int ls = 0; ls <= 9; ls += 3) {
        round8<true>(s, g, ls, chunk, log_n, w, ws, q, q2);
        __syncthreads();
      }
      for (uint32_t i = g; i < CHUNK; i += ROW_THREADS) ac[i] = s[i];
    }
    __syncthreads();
  }
  if (INV)
    for (uint32_t c = g; c < CHUNK; c += ROW_THREADS) column<N1, true>(a + c, w, ws, q, q2, ni, nis);
}

template <int N1, bool INV>
void launch_row(Ctx& c, size_t n_rows, uint64_t* base, const int16_t* pattern, int P) {
  ntt_row<N1, INV><<<(unsigned)n_rows, ROW_THREADS, 0, c.stream>>>(
      base, c.log_n, pattern, P, c.dmod(), static_cast<const uint64_t*>(INV ? c.d_itw.p : c.d_tw.p),
      static_cast<const uint64_t*>(INV ? c.d_itws.p : c.d_tws.p), c.d_ninv.u64(), c.d_ninvs.u64());
}

template <bool INV>
void ntt_run(Ctx& c, uint64_t* base, size_t n_rows, const int16_t* pattern, int P, size_t active) {
  if (n_rows == 0) return;
  const double bytes = 2.0 * (double)std::min(active, n_rows) * (double)c.N * 8.0;
  if (c.log_n <= CHUNK_LOG) {
    const int threads = std::min<int>(256, (int)(c.N / 2));
    Launch L_(c, K_NTT_SMALL, bytes);
    ntt_small<INV><<<(unsigned)n_rows, threads, c.N * 8, c.stream>>>(
        base, c.log_n, pattern, P, c.dmod(),
        static_cast<const uint64_t*>(INV ? c.d_itw.p : c.d_tw.p),
        static_cast<const uint64_t*>(INV ? c.d_itws.p : c.d_tws.p), c.d_ninv.u64(), c.d_ninvs.u64());
  } else {
    Launch L_(c, INV ? K_NTT_INV : K_NTT_FWD, bytes);
    switch (c.log_n - CHUNK_LOG) {
      case 1: launch_row<2, INV>(c, n_rows, base, pattern, P); break;
      case 2: launch_row<4, INV>(c, n_rows, base, pattern, P); break;
      case 3: launch_row<8, INV>(c, n_rows, base, pattern, P); break;
      case 4: launch_row<16, INV>(c, n_rows, base, pattern, P); break;
      default: throw Error(CKKS_ERR_UNSUPPORTED, "NTT size");
    }
  }
  CK_CUDA(cudaGetLastError());
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

}  // namespace ck
