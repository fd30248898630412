// ChaCha20 (RFC 8439) keystream and the samplers drawn from it.
//
// Stream (seed, domain, id): key = (seed lo, seed hi, 0 x 6), nonce =
// (domain, id lo, id hi); 32-bit word idx sits in block idx/16, word idx%16.
// Samplers: ternary s_i = (w32[i] mod 3) - 1 (domain 1, id 0);
// centred binomial e_i = popcount(w64[i] & (2^21-1)) - popcount((w64[i]>>21) &
// (2^21-1)) (domain 2); uniform a_t[i] = (w64[2i+1] 2^64 + w64[2i]) mod q_t
// (domain 3, id = object << 8 | t), w64[i] = w32[2i] | w32[2i+1] << 32.
// Sparse ternary of Hamming weight h (domain 4, id 0): a partial
// Fisher-Yates shuffle of 0..N-1, step i swapping position i with
// i + w32[2i] mod (N - i) and giving the coefficient at the position drawn
// the sign -1 if w32[2i+1] is odd, else +1.
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

__device__ __forceinline__ uint32_t rotl(uint32_t x, int r) { return __funnelshift_l(x, x, r); }

#define QROUND(a, b, c, d) \
  a += b; d ^= a; d = rotl(d, 16); \
  c += d; b ^= c; b = rotl(b, 12); \
  a += b; d ^= a; d = rotl(d, 8);  \
  c += d; b ^= c; b = rotl(b, 7);

__device__ void chacha_block(uint64_t seed, uint32_t domain, uint64_t id, uint32_t counter,
                             uint32_t out[16]) {
  uint32_t s[16];
  s[0] = 0x61707865u; s[1] = 0x3320646eu; s[2] = 0x79622d32u; s[3] = 0x6b206574u;
  s[4] = (uint32_t)seed; s[5] = (uint32_t)(seed >> 32);
  s[6] = s[7] = s[8] = s[9] = s[10] = s[11] = 0;
  s[12] = counter;
  s[13] = domain; s[14] = (uint32_t)id; s[15] = (uint32_t)(id >> 32);
  uint32_t x[16];
#pragma unroll
  for (int i = 0; i < 16; i++) x[i] = s[i];
#pragma unroll
  for (int r = 0; r < 10; r++) {
    QROUND(x[0], x[4], x[8], x[12]);
    QROUND(x[1], x[5], x[9], x[13]);
    QROUND(x[2], x[6], x[10], x[14]);
    QROUND(x[3], x[7], x[11], x[15]);
    QROUND(x[0], x[5], x[10], x[15]);
    QROUND(x[1], x[6], x[11], x[12]);
    QROUND(x[2], x[7], x[8], x[13]);
    QROUND(x[3], x[4], x[9], x[14]);
  }
#pragma unroll
  for (int i = 0; i < 16; i++) out[i] = x[i] + s[i];
}

// one block -> 16 coefficients
__global__ void ternary_kernel(uint64_t seed, int64_t* out, size_t N) {
  GRID_LOOP(blk, N / 16) {
    uint32_t w[16];
    chacha_block(seed, 1, 0, (uint32_t)blk, w);
#pragma unroll
    for (int k = 0; k < 16; k++) out[blk * 16 + k] = (int64_t)(w[k] % 3u) - 1;
  }
}

// one block -> 8 coefficients of object ids[o]
__global__ void cbd_kernel(uint64_t seed, const uint64_t* ids, size_t count, int64_t* out,
                           size_t N) {
  const size_t per = N / 8;
  GRID_LOOP(idx, count * per) {
    const size_t o = idx / per, blk = idx % per;
    uint32_t w[16];
    chacha_block(seed, 2, ids[o], (uint32_t)blk, w);
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const uint64_t v = (uint64_t)w[2 * k] | ((uint64_t)w[2 * k + 1] << 32);
      out[o * N + blk * 8 + k] =
          (int64_t)__popcll(v & 0x1FFFFFull) - (int64_t)__popcll((v >> 21) & 0x1FFFFFull);
    }
  }
}

// one block -> 4 coefficients of row r (modulus pattern[r]) of object ids[o]
__global__ void uniform_kernel(uint64_t seed, const uint64_t* ids, size_t count, int rows,
                               const int16_t* pattern, const Mod* mods, uint64_t* out, size_t N) {
  const size_t per = N / 4;
  GRID_LOOP(idx, count * rows * per) {
    const size_t blk = idx % per;
    const size_t orow = idx / per;
    const int r = (int)(orow % rows);
    const size_t o = orow / rows;
    const int t = pattern[r];
    const Mod m = mods[t];
    uint32_t w[16];
    chacha_block(seed, 3, (ids[o] << 8) | (uint64_t)t, (uint32_t)blk, w);
    const uint64_t two64 = (0 - m.q) % m.q;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint64_t lo = (uint64_t)w[4 * k] | ((uint64_t)w[4 * k + 1] << 32);
      const uint64_t hi = (uint64_t)w[4 * k + 2] | ((uint64_t)w[4 * k + 3] << 32);
      const uint64_t v = add_mod(mul_mod(hi % m.q, two64, m), lo % m.q, m.q);
      out[(o * rows + r) * N + blk * 4 + k] = v;
    }
  }
}

// the same stream as uniform_kernel for objects id_base + o; object o
// written at out + o * obj_rows * N (rows of another layout between objects)
__global__ void uniform_seq_kernel(uint64_t seed, uint64_t id_base, size_t count, int rows,
                                   const int16_t* pattern, const Mod* mods, uint64_t* out,
                                   size_t obj_rows, size_t N) {
  const size_t per = N / 4;
  GRID_LOOP(idx, count * rows * per) {
    const size_t blk = idx % per;
    const size_t orow = idx / per;
    const int r = (int)(orow % rows);
    const size_t o = orow / rows;
    const int t = pattern[r];
    const Mod m = mods[t];
    uint32_t w[16];
    chacha_block(seed, 3, ((id_base + o) << 8) | (uint64_t)t, (uint32_t)blk, w);
    const uint64_t two64 = (0 - m.q) % m.q;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint64_t lo = (uint64_t)w[4 * k] | ((uint64_t)w[4 * k + 1] << 32);
      const uint64_t hi = (uint64_t)w[4 * k + 2] | ((uint64_t)w[4 * k + 3] << 32);
      const uint64_t v = add_mod(mul_mod(hi % m.q, two64, m), lo % m.q, m.q);
      out[(o * obj_rows + r) * N + blk * 4 + k] = v;
    }
  }
}

__global__ void sparse_init_kernel(int64_t* s, uint32_t* perm, size_t N) {
  GRID_LOOP(i, N) {
    s[i] = 0;
    perm[i] = (uint32_t)i;
  }
}

// sequential by definition (each draw depends on the previous swaps); one thread
__global__ void sparse_shuffle_kernel(uint64_t seed, int h, int64_t* s, uint32_t* perm, size_t N) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  uint32_t w[16];
  uint32_t have = 0xFFFFFFFFu;
  for (int i = 0; i < h; i++) {
    uint32_t v[2];
    for (int k = 0; k < 2; k++) {
      const uint64_t idx = 2 * (uint64_t)i + k;
      if ((uint32_t)(idx / 16) != have) {
        have = (uint32_t)(idx / 16);
        chacha_block(seed, 4, 0, have, w);
      }
      v[k] = w[idx % 16];
    }
    const size_t j = (size_t)i + (size_t)(v[0] % (uint32_t)(N - (size_t)i));
    const uint32_t t = perm[i];
    perm[i] = perm[j];
    perm[j] = t;
    s[perm[i]] = (v[1] & 1u) ? -1 : 1;
  }
}

}  // namespace

void sample_sparse_ternary(Ctx& c, uint64_t seed, int h, int64_t* out) {
  if (h < 1 || (uint64_t)h > c.N) throw Error(CKKS_ERR_INVALID_ARG, "Hamming weight out of range");
  DevBuf perm(&c, c.N * 4);
  {
  Launch L_(c, K_SAMPLE, c.N * 12.0);
  sparse_init_kernel<<<grid_for(c.N), TPB, 0, c.stream>>>(out, static_cast<uint32_t*>(perm.p), c.N);
  CK_CUDA(cudaGetLastError());
  }
  Launch L_(c, K_SAMPLE, h * 24.0);
  sparse_shuffle_kernel<<<1, 32, 0, c.stream>>>(seed, h, out, static_cast<uint32_t*>(perm.p), c.N);
  CK_CUDA(cudaGetLastError());
}

void sample_ternary(Ctx& c, uint64_t seed, int64_t* out) {
  if (c.N < 16) throw Error(CKKS_ERR_UNSUPPORTED, "N < 16");
  Launch L_(c, K_SAMPLE, c.N * 8.0);
  ternary_kernel<<<grid_for(c.N / 16), TPB, 0, c.stream>>>(seed, out, c.N);
  CK_CUDA(cudaGetLastError());
}

void sample_cbd(Ctx& c, uint64_t seed, const uint64_t* ids, size_t count, int64_t* out) {
  Launch L_(c, K_SAMPLE, count * c.N * 8.0);
  cbd_kernel<<<grid_for(count * c.N / 8), TPB, 0, c.stream>>>(seed, ids, count, out, c.N);
  CK_CUDA(cudaGetLastError());
}

void sample_uniform_seq(Ctx& c, uint64_t seed, uint64_t id_base, size_t count, int rows,
                        const int16_t* pattern, uint64_t* out, size_t obj_rows) {
  Launch L_(c, K_SAMPLE, count * rows * c.N * 8.0);
  uniform_seq_kernel<<<grid_for(count * rows * c.N / 4), TPB, 0, c.stream>>>(
      seed, id_base, count, rows, pattern, c.dmod(), out, obj_rows, c.N);
  CK_CUDA(cudaGetLastError());
}

void sample_uniform(Ctx& c, uint64_t seed, const uint64_t* ids, size_t count, int rows,
                    const int16_t* pattern, uint64_t* out) {
  Launch L_(c, K_SAMPLE, count * rows * c.N * 8.0);
  uniform_kernel<<<grid_for(count * rows * c.N / 4), TPB, 0, c.stream>>>(
      seed, ids, count, rows, pattern, c.dmod(), out, c.N);
  CK_CUDA(cudaGetLastError());
}

}  // namespace ck
