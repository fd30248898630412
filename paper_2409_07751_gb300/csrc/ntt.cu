// Batched negacyclic NTT / inverse NTT over uint64 residues.
//
// Forward map (bit-reversed output): A[j] = sum_i a[i] psi^((2 brv(j)+1) i),
// computed by radix-2 Cooley-Tukey stages m = 1, 2, ..., N/2 where block i
// of stage m uses the twiddle psi^brv(m+i) (the psi twist merged into the
// twiddles). The inverse runs Gentleman-Sande stages m = N/2, ..., 1 with
// psi^-brv(m+i), then scales by N^-1.
//
// N <= 4096: one CTA holds a row in shared memory.
// N >= 8192: N = N1 * N2 with N2 = 4096. The first log2(N1) forward stages
// only couple elements c + s*N2 (s < N1) of one column c, so each thread
// transforms one column in registers (coalesced across the warp); the
// remaining log2(N2) stages stay inside contiguous chunks of N2 elements,
// which one CTA transforms in shared memory. The inverse runs the same two
// phases in the opposite order.
#include <algorithm>

#include "modarith.cuh"

namespace ck {

namespace {

constexpr int CHUNK_LOG = 12;
constexpr int CHUNK = 1 << CHUNK_LOG;  // N2
constexpr int CHUNK_THREADS = 512;

struct TwTab {
  const uint64_t* w;
  const uint64_t* ws;
};

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
    for (uint32_t m = 1, t = half; m < N; m <<= 1, t >>= 1) {
      for (uint32_t k = threadIdx.x; k < half; k += blockDim.x) {
        const uint32_t ib = k / t, jj = k % t, j = ib * 2 * t + jj;
        ct_bfly(sm[j], sm[j + t], w[m + ib], ws[m + ib], q);
      }
      __syncthreads();
    }
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) a[i] = sm[i];
  } else {
    for (uint32_t m = half, t = 1; m >= 1; m >>= 1, t <<= 1) {
      for (uint32_t k = threadIdx.x; k < half; k += blockDim.x) {
        const uint32_t ib = k / t, jj = k % t, j = ib * 2 * t + jj;
        gs_bfly(sm[j], sm[j + t], w[m + ib], ws[m + ib], q);
      }
      __syncthreads();
    }
    const uint64_t ni = ninv[mi], nis = ninvs[mi];
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) a[i] = mul_shoup(sm[i], ni, nis, q);
  }
}

// ---------------------------------------------------------------- phase: columns
template <int N1, bool INV>
__global__ void ntt_columns(uint64_t* base, int log_n, const int16_t* pattern, int P,
                            const Mod* mods, const uint64_t* tw, const uint64_t* tws,
                            const uint64_t* ninv, const uint64_t* ninvs) {
  constexpr int PER_ROW = CHUNK / 256;  // blocks per row
  const size_t row = blockIdx.x / PER_ROW;
  const int mi = pattern[row % P];
  if (mi < 0) return;
  const uint32_t c = (blockIdx.x % PER_ROW) * 256 + threadIdx.x;
  const size_t N = (size_t)1 << log_n;
  const uint64_t q = mods[mi].q;
  const uint64_t* w = tw + (size_t)mi * N;
  const uint64_t* ws = tws + (size_t)mi * N;
  uint64_t* a = base + row * N + c;
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
        for (int jj = 0; jj < t1; jj++) ct_bfly(x[i * 2 * t1 + jj], x[i * 2 * t1 + jj + t1], wv, wsv, q);
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
        for (int jj = 0; jj < t1; jj++) gs_bfly(x[i * 2 * t1 + jj], x[i * 2 * t1 + jj + t1], wv, wsv, q);
      }
    }
    const uint64_t ni = ninv[mi], nis = ninvs[mi];
#pragma unroll
    for (int s = 0; s < N1; s++) a[(size_t)s * CHUNK] = mul_shoup(x[s], ni, nis, q);
  }
}

// ---------------------------------------------------------------- phase: chunks
template <bool INV>
__global__ void __launch_bounds__(CHUNK_THREADS) ntt_chunks(uint64_t* base, int log_n,
                                                            const int16_t* pattern, int P,
                                                            const Mod* mods, const uint64_t* tw,
                                                            const uint64_t* tws) {
  __shared__ uint64_t sm[CHUNK];
  const uint32_t N1 = 1u << (log_n - CHUNK_LOG);
  const size_t row = blockIdx.x / N1;
  const int mi = pattern[row % P];
  if (mi < 0) return;
  const uint32_t b = blockIdx.x % N1;
  const size_t N = (size_t)1 << log_n;
  const uint64_t q = mods[mi].q;
  const uint64_t* w = tw + (size_t)mi * N;
  const uint64_t* ws = tws + (size_t)mi * N;
  uint64_t* a = base + row * N + (size_t)b * CHUNK;
  for (int i = threadIdx.x; i < CHUNK; i += CHUNK_THREADS) sm[i] = a[i];
  __syncthreads();
  const uint32_t NN = (uint32_t)N;
  if (!INV) {
    for (uint32_t m = N1, t = CHUNK / 2; m < NN; m <<= 1, t >>= 1) {
      const uint32_t blocks_per_chunk = CHUNK / (2 * t);
      for (uint32_t k = threadIdx.x; k < CHUNK / 2; k += CHUNK_THREADS) {
        const uint32_t ib = k / t, jj = k % t, j = ib * 2 * t + jj;
        const uint32_t ig = m + b * blocks_per_chunk + ib;
        ct_bfly(sm[j], sm[j + t], w[ig], ws[ig], q);
      }
      __syncthreads();
    }
  } else {
    for (uint32_t m = NN / 2, t = 1; m >= N1; m >>= 1, t <<= 1) {
      const uint32_t blocks_per_chunk = CHUNK / (2 * t);
      for (uint32_t k = threadIdx.x; k < CHUNK / 2; k += CHUNK_THREADS) {
        const uint32_t ib = k / t, jj = k % t, j = ib * 2 * t + jj;
        const uint32_t ig = m + b * blocks_per_chunk + ib;
        gs_bfly(sm[j], sm[j + t], w[ig], ws[ig], q);
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < CHUNK; i += CHUNK_THREADS) a[i] = sm[i];
}

template <bool INV>
void launch_columns(int N1, dim3 g, cudaStream_t s, uint64_t* base, int log_n,
                    const int16_t* pattern, int P, const Mod* mods, const uint64_t* tw,
                    const uint64_t* tws, const uint64_t* ni, const uint64_t* nis) {
  switch (N1) {
    case 2: ntt_columns<2, INV><<<g, 256, 0, s>>>(base, log_n, pattern, P, mods, tw, tws, ni, nis); break;
    case 4: ntt_columns<4, INV><<<g, 256, 0, s>>>(base, log_n, pattern, P, mods, tw, tws, ni, nis); break;
    case 8: ntt_columns<8, INV><<<g, 256, 0, s>>>(base, log_n, pattern, P, mods, tw, tws, ni, nis); break;
    case 16: ntt_columns<16, INV><<<g, 256, 0, s>>>(base, log_n, pattern, P, mods, tw, tws, ni, nis); break;
    default: throw Error(CKKS_ERR_UNSUPPORTED, "NTT size");
  }
}

template <bool INV>
void ntt_run(Ctx& c, uint64_t* base, size_t n_rows, const int16_t* pattern, int P, size_t active) {
  if (n_rows == 0) return;
  const double bytes = 2.0 * (double)std::min(active, n_rows) * (double)c.N * 8.0;
  const Mod* mods = c.dmod();
  const uint64_t* tw = static_cast<const uint64_t*>(INV ? c.d_itw.p : c.d_tw.p);
  const uint64_t* tws = static_cast<const uint64_t*>(INV ? c.d_itws.p : c.d_tws.p);
  const uint64_t* ni = static_cast<const uint64_t*>(c.d_ninv.p);
  const uint64_t* nis = static_cast<const uint64_t*>(c.d_ninvs.p);
  if (c.log_n <= CHUNK_LOG) {
    const int threads = std::min<int>(256, (int)(c.N / 2));
    Launch L_(c, K_NTT_SMALL, bytes);
    ntt_small<INV><<<(unsigned)n_rows, threads, c.N * 8, c.stream>>>(base, c.log_n, pattern, P,
                                                                     mods, tw, tws, ni, nis);
  } else {
    const int N1 = 1 << (c.log_n - CHUNK_LOG);
    const dim3 gcol((unsigned)(n_rows * (CHUNK / 256)));
    const dim3 gchk((unsigned)(n_rows * N1));
    if (!INV) {
      {
        Launch L_(c, K_NTT_FWD_COL, bytes);
        launch_columns<false>(N1, gcol, c.stream, base, c.log_n, pattern, P, mods, tw, tws, ni, nis);
      }
      Launch L_(c, K_NTT_FWD_CHUNK, bytes);
      ntt_chunks<false><<<gchk, CHUNK_THREADS, 0, c.stream>>>(base, c.log_n, pattern, P, mods, tw, tws);
    } else {
      {
        Launch L_(c, K_NTT_INV_CHUNK, bytes);
        ntt_chunks<true><<<gchk, CHUNK_THREADS, 0, c.stream>>>(base, c.log_n, pattern, P, mods, tw, tws);
      }
      Launch L_(c, K_NTT_INV_COL, bytes);
      launch_columns<true>(N1, gcol, c.stream, base, c.log_n, pattern, P, mods, tw, tws, ni, nis);
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
