// Integer-pipe peaks of this GPU, measured: the denominators of the integer
// roofline that the NTT kinds are reported against.
//
// Every thread runs CHAINS independent dependency chains on register values
// (no memory traffic inside the timed loop) of one of:
//   kind 0: a 64 x 64 -> 128-bit product (the low and high words);
//   kind 1: the forward transform's lazy butterfly (ct_grow: a three-product
//           Shoup multiply plus the two 64-bit sums, as the transforms run
//           it), 16 stages then the full
//           reduction of both words, the ratio of butterflies to reductions
//           of a 2^16-point transform;
//   kind 2: the three-product Shoup multiply alone (the basis-conversion
//           product of ModUp and ModDown), accumulated lazily;
//   kind 3: kind 1 with the remainder formed as y w - Q q on 64-bit words
//           (the form the transforms used before the one-chain remainder);
//   kind 4: kind 1 where every butterfly takes its partner word from another
//           lane through two 32-bit warp shuffles (the exchange of a
//           shuffle-based transform);
//   kind 5: kind 1 where the partner word goes through shared memory (a
//           store, a block barrier and a load per stage, the exchange of the
//           shared-memory rounds).
// The grid is the SM count times the resident blocks per SM; the rate is the
// operations of several launches over their CUDA-event time, after a warm-up
// launch, on the context's stream.
#include <algorithm>

#include "modarith.cuh"
#include "ops.h"

using namespace ck;

namespace {

constexpr int PEAK_THREADS = 256;
constexpr int CHAINS = 8;

template <int KIND>
__global__ void __launch_bounds__(PEAK_THREADS) k_int_peak(uint64_t* out, uint64_t q, uint64_t w,
                                                           uint64_t ws, uint64_t w1s, int iters) {
  const uint64_t t0 = blockIdx.x * (uint64_t)PEAK_THREADS + threadIdx.x;
  uint64_t x[CHAINS], y[CHAINS];
#pragma unroll
  for (int j = 0; j < CHAINS; j++) {
    x[j] = (t0 * 0x9E3779B97F4A7C15ull + j) % q;
    y[j] = (t0 * 0xC2B2AE3D27D4EB4Full + 7 * j + 1) % q;
  }
  const uint64_t q2 = 2 * q;
  for (int it = 0; it < iters; it++) {
    if (KIND == 0) {
#pragma unroll
      for (int j = 0; j < CHAINS; j++) {
        const uint64_t lo = x[j] * y[j], hi = __umul64hi(x[j], y[j]);
        x[j] = lo ^ hi;
        y[j] += 0x9E3779B97F4A7C15ull;
      }
    } else if (KIND == 1) {
#pragma unroll
      for (int s = 0; s < 16; s++) {
#pragma unroll
        for (int j = 0; j < CHAINS; j++) ct_grow(x[j], y[j], w, ws, q, q2);
      }
#pragma unroll
      for (int j = 0; j < CHAINS; j++) {
        x[j] = reduce_full(x[j], q, w1s);
        y[j] = reduce_full(y[j], q, w1s);
      }
    } else if (KIND == 2) {
#pragma unroll
      for (int s = 0; s < 16; s++) {
#pragma unroll
        for (int j = 0; j < CHAINS; j++) x[j] = shoup_approx(x[j], w, ws, q) + y[j];
      }
#pragma unroll
      for (int j = 0; j < CHAINS; j++) x[j] = reduce_full(x[j], q, w1s);
    } else if (KIND == 3) {
#pragma unroll
      for (int s = 0; s < 16; s++) {
#pragma unroll
        for (int j = 0; j < CHAINS; j++) {
          const uint64_t u = x[j];
          const uint64_t t = shoup_approx_sub(y[j], w, ws, q);
          x[j] = u + t;
          y[j] = u - t + 2 * q2;
        }
      }
#pragma unroll
      for (int j = 0; j < CHAINS; j++) {
        x[j] = reduce_full(x[j], q, w1s);
        y[j] = reduce_full(y[j], q, w1s);
      }
    } else if (KIND == 4) {
      // lane pairs (lane, lane ^ 1): the even lane keeps x, the odd lane y
      const bool hi_lane = threadIdx.x & 1;
#pragma unroll
      for (int s = 0; s < 16; s++) {
#pragma unroll
        for (int j = 0; j < CHAINS; j++) {
          const uint64_t mine = hi_lane ? y[j] : x[j];
          const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)mine, 1);
          const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(mine >> 32), 1);
          const uint64_t other = ((uint64_t)hi << 32) | lo;
          uint64_t a = hi_lane ? other : mine, b = hi_lane ? mine : other;
          ct_grow(a, b, w, ws, q, q2);
          if (hi_lane) y[j] = b; else x[j] = a;
        }
      }
#pragma unroll
      for (int j = 0; j < CHAINS; j++) {
        x[j] = reduce_full(x[j], q, w1s);
        y[j] = reduce_full(y[j], q, w1s);
      }
    } else {
      __shared__ uint64_t xs[PEAK_THREADS * CHAINS];
      const bool hi_lane = threadIdx.x & 1;
#pragma unroll
      for (int s = 0; s < 16; s++) {
#pragma unroll
        for (int j = 0; j < CHAINS; j++) xs[j * PEAK_THREADS + threadIdx.x] = hi_lane ? y[j] : x[j];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < CHAINS; j++) {
          const uint64_t other = xs[j * PEAK_THREADS + (threadIdx.x ^ 1)];
          const uint64_t mine = hi_lane ? y[j] : x[j];
          uint64_t a = hi_lane ? other : mine, b = hi_lane ? mine : other;
          ct_grow(a, b, w, ws, q, q2);
          if (hi_lane) y[j] = b; else x[j] = a;
        }
        __syncthreads();
      }
#pragma unroll
      for (int j = 0; j < CHAINS; j++) {
        x[j] = reduce_full(x[j], q, w1s);
        y[j] = reduce_full(y[j], q, w1s);
      }
    }
  }
  uint64_t f = 0;
#pragma unroll
  for (int j = 0; j < CHAINS; j++) f ^= x[j] + y[j];
  out[t0] = f;  // keeps every chain live
}

template <int KIND>
double run_peak(Ctx& c, uint64_t* out, int blocks, uint64_t q, uint64_t w, uint64_t ws,
                uint64_t w1s) {
  constexpr int ITERS = KIND == 0 ? 4096 : 256;
  // kinds 4 and 5: a lane pair computes each butterfly on both lanes
  constexpr double OPS_PER_ITER = KIND == 0 ? CHAINS : (KIND >= 4 ? 8.0 : 16.0) * CHAINS;
  constexpr int REPS = 5;
  k_int_peak<KIND><<<blocks, PEAK_THREADS, 0, c.stream>>>(out, q, w, ws, w1s, ITERS);
  CK_CUDA(cudaGetLastError());
  cudaEvent_t a, b;
  CK_CUDA(cudaEventCreate(&a));
  CK_CUDA(cudaEventCreate(&b));
  CK_CUDA(cudaEventRecord(a, c.stream));
  for (int r = 0; r < REPS; r++)
    k_int_peak<KIND><<<blocks, PEAK_THREADS, 0, c.stream>>>(out, q, w, ws, w1s, ITERS);
  CK_CUDA(cudaEventRecord(b, c.stream));
  CK_CUDA(cudaEventSynchronize(b));
  float ms = 0.f;
  CK_CUDA(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  const double ops = (double)REPS * blocks * PEAK_THREADS * ITERS * OPS_PER_ITER;
  return ops / (ms / 1000.0);
}

}  // namespace

extern "C" int ckks_int_peak(ckks_ctx* ctx, int kind, double* per_s) {
  try {
    if (!ctx || !per_s || kind < 0 || kind > 5) return CKKS_ERR_INVALID_ARG;
    Ctx& c = ctx->c;
    CK_CUDA(cudaSetDevice(c.device));
    int sms = 0, per_sm = 0;
    CK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device));
    auto occ = [&](auto kernel) {
      CK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, PEAK_THREADS, 0));
    };
    switch (kind) {
      case 0: occ(k_int_peak<0>); break;
      case 1: occ(k_int_peak<1>); break;
      case 2: occ(k_int_peak<2>); break;
      case 3: occ(k_int_peak<3>); break;
      case 4: occ(k_int_peak<4>); break;
      default: occ(k_int_peak<5>); break;
    }
    const int blocks = sms * std::max(per_sm, 1);
    // a rescaling prime of the chain (40 bits), as in the transforms that dominate
    const int t = c.L >= 1 ? 1 : 0;
    const uint64_t q = c.mod[t];
    const uint64_t w = c.psi[t] % q;
    const uint64_t ws = shoup_h(w, q), w1s = shoup_h(1, q);
    DevBuf out(&c, (size_t)blocks * PEAK_THREADS * 8);
    double r = 0.0;
    switch (kind) {
      case 0: r = run_peak<0>(c, out.u64(), blocks, q, w, ws, w1s); break;
      case 1: r = run_peak<1>(c, out.u64(), blocks, q, w, ws, w1s); break;
      case 2: r = run_peak<2>(c, out.u64(), blocks, q, w, ws, w1s); break;
      case 3: r = run_peak<3>(c, out.u64(), blocks, q, w, ws, w1s); break;
      case 4: r = run_peak<4>(c, out.u64(), blocks, q, w, ws, w1s); break;
      default: r = run_peak<5>(c, out.u64(), blocks, q, w, ws, w1s); break;
    }
    *per_s = r;
    return CKKS_OK;
  } catch (...) {
    return api_error();
  }
}
