// Canonical-embedding encoder / decoder in FP64.
//
// Slots: n = N/2, slot j <-> zeta^(5^j mod 2N), zeta = exp(i pi / N). With
// w_i = m_i + i m_{i+n}, slot j = sum_i (w_i zeta^i) omega^(k_j i),
// omega = zeta^4, k_j = (5^j mod 2N - 1)/4. Encoding places z_j at k_j, runs
// an inverse radix-2 DFT (decimation in time on bit-reversed input, twiddle
// T[4 t n/len] conjugated), untwists by zeta^-i, scales by S/n and rounds
// half-to-even. Every butterfly is evaluated in a fixed order with no fused
// multiply-add (the library is compiled with -fmad=false), so the integers
// are the same as those of any IEEE-754 evaluation of the same steps.
#include "modarith.cuh"

namespace ck {

void k_int_to_rns(Ctx& c, const int64_t* v, uint64_t* out, size_t polys, int rows,
                  const int16_t* pattern);

namespace {

constexpr int TPB = 256;
inline unsigned grid_for(size_t total) {
  size_t g = (total + TPB - 1) / TPB;
  const size_t cap = 152 * 32;
  return (unsigned)(g < cap ? (g ? g : 1) : cap);
}
#define GRID_LOOP(idx, total) \
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (total); idx += (size_t)gridDim.x * blockDim.x)

__device__ __forceinline__ uint32_t brv(uint32_t x, int bits) { return __brev(x) >> (32 - bits); }

__global__ void place_kernel(const double* v, const double* vi, size_t nv, double* xr, double* xi,
                             size_t B, int log_n, const uint32_t* slot) {
  const size_t n = (size_t)1 << (log_n - 1);
  GRID_LOOP(idx, B * nv) {
    const size_t b = idx / nv, j = idx % nv;
    const size_t p = b * n + brv(slot[j], log_n - 1);
    xr[p] = v[idx];
    if (vi) xi[p] = vi[idx];
  }
}

// one radix-2 stage of length `len` on B transforms of n points
__global__ void stage_kernel(double* xr, double* xi, size_t B, int log_n, uint32_t len,
                             const double* T, int sign) {
  const size_t n = (size_t)1 << (log_n - 1);
  const uint32_t half = len >> 1;
  const uint32_t step = (uint32_t)(n / len);
  GRID_LOOP(idx, B * (n / 2)) {
    const size_t b = idx / (n / 2);
    const uint32_t k = (uint32_t)(idx % (n / 2));
    const uint32_t s = (k / half) * len, t = k % half;
    const uint32_t ti = 4u * t * step;
    const double wr = T[2 * ti];
    const double wi = sign > 0 ? T[2 * ti + 1] : -T[2 * ti + 1];
    double* r = xr + b * n;
    double* im = xi + b * n;
    const double br = r[s + t + half], bi = im[s + t + half];
    const double pr = br * wr - bi * wi;
    const double pi = br * wi + bi * wr;
    const double ar = r[s + t], ai = im[s + t];
    r[s + t] = ar + pr;
    im[s + t] = ai + pi;
    r[s + t + half] = ar - pr;
    im[s + t + half] = ai - pi;
  }
}

__global__ void untwist_round_kernel(const double* xr, const double* xi, int64_t* out, size_t B,
                                     int log_n, const double* T, double f, int* flag) {
  const size_t n = (size_t)1 << (log_n - 1);
  const size_t N = 2 * n;
  GRID_LOOP(idx, B * n) {
    const size_t b = idx / n, i = idx % n;
    const double tr = T[2 * i], ti = T[2 * i + 1];
    const double re = xr[idx] * tr + xi[idx] * ti;
    const double im = xi[idx] * tr - xr[idx] * ti;
    const double a = rint(re * f), c = rint(im * f);
    if (!(fabs(a) < 9.2e18) || !(fabs(c) < 9.2e18)) {
      atomicExch(flag, 1);
      out[b * N + i] = 0;
      out[b * N + i + n] = 0;
    } else {
      out[b * N + i] = (int64_t)a;
      out[b * N + i + n] = (int64_t)c;
    }
  }
}

// decode input: m[b][N] residues mod q0 -> twisted values at bit-reversed positions
__global__ void twist_kernel(const uint64_t* m, double* xr, double* xi, size_t B, int log_n,
                             uint64_t q0, double scale, const double* T) {
  const size_t n = (size_t)1 << (log_n - 1);
  const size_t N = 2 * n;
  GRID_LOOP(idx, B * n) {
    const size_t b = idx / n, i = idx % n;
    const uint64_t x0 = m[b * N + i], x1 = m[b * N + i + n];
    const int64_t v0 = x0 > q0 / 2 ? -(int64_t)(q0 - x0) : (int64_t)x0;
    const int64_t v1 = x1 > q0 / 2 ? -(int64_t)(q0 - x1) : (int64_t)x1;
    const double mr = (double)v0 / scale, mi = (double)v1 / scale;
    const double tr = T[2 * i], ti = T[2 * i + 1];
    const size_t p = b * n + brv((uint32_t)i, log_n - 1);
    xr[p] = mr * tr - mi * ti;
    xi[p] = mr * ti + mi * tr;
  }
}

__global__ void gather_kernel(const double* xr, double* out, size_t B, size_t nv, int log_n,
                              const uint32_t* slot) {
  const size_t n = (size_t)1 << (log_n - 1);
  GRID_LOOP(idx, B * nv) {
    const size_t b = idx / nv, j = idx % nv;
    out[idx] = xr[b * n + slot[j]];
  }
}

void run_stages(Ctx& c, double* xr, double* xi, size_t B, int sign) {
  const size_t n = c.N / 2;
  for (uint32_t len = 2; len <= n; len <<= 1) {
    Launch L_(c, K_ENCODE, 8.0 * B * n * 8);
    stage_kernel<<<grid_for(B * (n / 2)), TPB, 0, c.stream>>>(
        xr, xi, B, c.log_n, len, static_cast<const double*>(c.d_fft.p), sign);
  }
  CK_CUDA(cudaGetLastError());
}

}  // namespace

int encode(Ctx& c, const double* d_v, size_t B, size_t nv, int level, double scale, uint64_t* pt) {
  return encode_rows(c, d_v, B, nv, level + 1, c.iota(), scale, pt);
}

int encode_rows(Ctx& c, const double* d_v, size_t B, size_t nv, int rows, const int16_t* pattern,
                double scale, uint64_t* pt, const double* d_im) {
  const size_t n = c.N / 2;
  if (nv > n) throw Error(CKKS_ERR_INVALID_ARG, "more values than slots");
  DevBuf xr(&c, B * n * 8), xi(&c, B * n * 8), coef(&c, B * c.N * 8);
  CK_CUDA(cudaMemsetAsync(xr.p, 0, xr.bytes, c.stream));
  CK_CUDA(cudaMemsetAsync(xi.p, 0, xi.bytes, c.stream));
  CK_CUDA(cudaMemsetAsync(c.d_flag.p, 0, 4, c.stream));
  if (nv) {
    Launch L_(c, K_ENCODE, 2.0 * B * nv * 8);
    place_kernel<<<grid_for(B * nv), TPB, 0, c.stream>>>(
        d_v, d_im, nv, static_cast<double*>(xr.p), static_cast<double*>(xi.p), B, c.log_n,
        static_cast<const uint32_t*>(c.d_slot.p));
  }
  run_stages(c, static_cast<double*>(xr.p), static_cast<double*>(xi.p), B, -1);
  const double f = scale / (double)n;
  {
  Launch L_(c, K_ENCODE, 4.0 * B * n * 8);
  untwist_round_kernel<<<grid_for(B * n), TPB, 0, c.stream>>>(
      static_cast<double*>(xr.p), static_cast<double*>(xi.p), static_cast<int64_t*>(coef.p), B,
      c.log_n, static_cast<const double*>(c.d_fft.p), f, static_cast<int*>(c.d_flag.p));
  CK_CUDA(cudaGetLastError());
  }
  k_int_to_rns(c, static_cast<int64_t*>(coef.p), pt, B, rows, pattern);
  ntt_forward(c, pt, B * rows, pattern, rows);
  int flag = 0;
  CK_CUDA(cudaMemcpyAsync(&flag, c.d_flag.p, 4, cudaMemcpyDeviceToHost, c.stream));
  CK_CUDA(cudaStreamSynchronize(c.stream));
  return flag ? CKKS_ERR_OVERFLOW : CKKS_OK;
}

void decode_limb0(Ctx& c, const uint64_t* m, size_t B, double scale, double* d_out, size_t nv) {
  const size_t n = c.N / 2;
  DevBuf xr(&c, B * n * 8), xi(&c, B * n * 8);
  {
  Launch L_(c, K_ENCODE, 4.0 * B * n * 8);
  twist_kernel<<<grid_for(B * n), TPB, 0, c.stream>>>(m, static_cast<double*>(xr.p),
                                                      static_cast<double*>(xi.p), B, c.log_n,
                                                      c.mod[0], scale,
                                                      static_cast<const double*>(c.d_fft.p));
  CK_CUDA(cudaGetLastError());
  }
  run_stages(c, static_cast<double*>(xr.p), static_cast<double*>(xi.p), B, +1);
  Launch L_(c, K_ENCODE, 2.0 * B * nv * 8);
  gather_kernel<<<grid_for(B * nv), TPB, 0, c.stream>>>(static_cast<double*>(xr.p), d_out, B, nv,
                                                        c.log_n,
                                                        static_cast<const uint32_t*>(c.d_slot.p));
  CK_CUDA(cudaGetLastError());
}

}  // namespace ck
