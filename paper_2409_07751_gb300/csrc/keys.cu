// Key generation, encryption and decryption.
//
// Secret s: ternary (dense, or sparse of a given Hamming weight), NTT form
// over every QP modulus. Switching key from s'
// to s for digit j and modulus t: b = e - a s + [t in D_j] [P]_{q_t} s',
// a uniform; s' = s^2 (relinearisation) or sigma_g(s) (Galois element g);
// randomness from object id 2^40 | g << 8 | j. Encryption at level l:
// c0 = m - a s + e, c1 = a with object id first_index + b.
#include "modarith.cuh"
#include "ops.h"

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

// key[j][0][t] = e[j][t] - key[j][1][t] * s[t] + (t <= L && t / alpha == j) Pmod[t] sp[t]
__global__ void keygen_b_kernel(uint64_t* key, const uint64_t* e, const uint64_t* s,
                                const uint64_t* sp, const uint64_t* pmod, int beta, int n_qp,
                                int L, int alpha, int log_n, const Mod* mods) {
  const size_t N = (size_t)1 << log_n;
  GRID_LOOP(idx, (size_t)beta * n_qp * N) {
    const size_t n = idx & (N - 1);
    const size_t jt = idx >> log_n;
    const int t = (int)(jt % n_qp);
    const int j = (int)(jt / n_qp);
    const Mod m = mods[t];
    const uint64_t a = key[(((size_t)j * 2 + 1) * n_qp + t) * N + n];
    uint64_t v = sub_mod(e[idx], mul_mod(a, s[(size_t)t * N + n], m), m.q);
    if (t <= L && t / alpha == j) v = add_mod(v, mul_mod(pmod[t], sp[(size_t)t * N + n], m), m.q);
    key[(((size_t)j * 2 + 0) * n_qp + t) * N + n] = v;
  }
}

// ct[b][0][t] = m[b][t] - a s + e ; ct[b][1][t] = a  (a, e, m: [B][l][N])
__global__ void encrypt_kernel(uint64_t* ct, const uint64_t* m, const uint64_t* a,
                               const uint64_t* e, const uint64_t* s, size_t B, int l, int log_n,
                               const Mod* mods) {
  const size_t N = (size_t)1 << log_n;
  const size_t per = (size_t)l * N;
  GRID_LOOP(idx, B * per) {
    const size_t b = idx / per, r = idx % per;
    const int t = (int)(r >> log_n);
    const Mod mm = mods[t];
    const uint64_t av = a[idx];
    const uint64_t v = add_mod(sub_mod(m[idx], mul_mod(av, s[r], mm), mm.q), e[idx], mm.q);
    ct[b * 2 * per + r] = v;
    ct[b * 2 * per + per + r] = av;
  }
}

// x[b][n] = c0[b][0][n] + c1[b][0][n] * s[0][n]
__global__ void decrypt_limb0_kernel(const uint64_t* ct, const uint64_t* s, uint64_t* x, size_t B,
                                     int l, int log_n, const Mod* mods) {
  const size_t N = (size_t)1 << log_n;
  GRID_LOOP(idx, B * N) {
    const size_t b = idx >> log_n, n = idx & (N - 1);
    const Mod m = mods[0];
    const uint64_t c0 = ct[b * 2 * l * N + n], c1 = ct[(b * 2 + 1) * l * N + n];
    x[idx] = add_mod(c0, mul_mod(c1, s[n], m), m.q);
  }
}

std::unique_ptr<DevBuf> switch_key(Ctx& c, const ckks_keys& k, uint64_t seed, uint64_t g,
                                   const int64_t* s_coef_dev) {
  const uint64_t a_seed = k.own_a_seed ? k.a_seed : seed;
  (void)s_coef_dev;
  const size_t N = c.N;
  const int beta = c.beta_max, n_qp = c.n_qp;
  DevBuf sp(&c, (size_t)n_qp * N * 8);
  if (g == 0)
    k_mul_pt(c, k.s.u64(), k.s.u64(), sp.u64(), n_qp, n_qp);
  else
    k_automorphism(c, k.s.u64(), sp.u64(), n_qp, c.perm(g));
  std::vector<uint64_t> ids(beta);
  for (int j = 0; j < beta; j++) ids[j] = (1ull << 40) | (g << 8) | (uint64_t)j;
  DevBuf d_ids(&c, beta * 8);
  CK_CUDA(cudaMemcpyAsync(d_ids.p, ids.data(), beta * 8, cudaMemcpyHostToDevice, c.stream));
  DevBuf e(&c, (size_t)beta * N * 8), er(&c, (size_t)beta * n_qp * N * 8);
  sample_cbd(c, seed, d_ids.u64(), beta, static_cast<int64_t*>(e.p));
  k_int_to_rns(c, static_cast<int64_t*>(e.p), er.u64(), beta, n_qp, c.iota());
  ntt_forward(c, er.u64(), (size_t)beta * n_qp, c.iota(), n_qp);
  auto key = std::make_unique<DevBuf>(&c, (size_t)beta * 2 * n_qp * N * 8);
  DevBuf a(&c, (size_t)beta * n_qp * N * 8);
  sample_uniform(c, a_seed, d_ids.u64(), beta, n_qp, c.iota(), a.u64());
  CK_CUDA(cudaMemcpy2DAsync(key->u64() + (size_t)n_qp * N, 2 * (size_t)n_qp * N * 8, a.p,
                            (size_t)n_qp * N * 8, (size_t)n_qp * N * 8, beta,
                            cudaMemcpyDeviceToDevice, c.stream));
  {
  Launch L_(c, K_CRYPT, 5.0 * beta * n_qp * N * 8);
  keygen_b_kernel<<<grid_for((size_t)beta * n_qp * N), TPB, 0, c.stream>>>(
      key->u64(), er.u64(), k.s.u64(), sp.u64(), c.d_pmod.u64(), beta, n_qp, c.L, c.alpha, c.log_n,
      c.dmod());
  CK_CUDA(cudaGetLastError());
  }
  return key;
}

}  // namespace

std::unique_ptr<ckks_keys> keygen(Ctx& c, uint64_t seed, const std::vector<int64_t>& steps,
                                  int hamming, bool conjugation, uint64_t a_seed) {
  auto k = std::make_unique<ckks_keys>();
  k->ctx = &c;
  k->a_seed = a_seed ? a_seed : seed;
  k->own_a_seed = a_seed != 0;
  const size_t N = c.N;
  DevBuf sc(&c, N * 8);
  if (hamming > 0)
    sample_sparse_ternary(c, seed, hamming, static_cast<int64_t*>(sc.p));
  else
    sample_ternary(c, seed, static_cast<int64_t*>(sc.p));
  k->s = DevBuf(&c, (size_t)c.n_qp * N * 8);
  k_int_to_rns(c, static_cast<int64_t*>(sc.p), k->s.u64(), 1, c.n_qp, c.iota());
  ntt_forward(c, k->s.u64(), c.n_qp, c.iota(), c.n_qp);
  k->relin = std::move(*switch_key(c, *k, seed, 0, nullptr));
  for (int64_t t : steps) {
    const uint64_t g = c.galois(t);
    if (g == 1 || k->galois.count(g)) continue;
    k->galois[g] = switch_key(c, *k, seed, g, nullptr);
  }
  if (conjugation) k->galois[2 * N - 1] = switch_key(c, *k, seed, 2 * N - 1, nullptr);
  CK_CUDA(cudaStreamSynchronize(c.stream));
  return k;
}

const uint64_t* switch_key_words(Ctx& c, const ckks_keys& keys, uint64_t g, DevBuf& tmp) {
  const DevBuf* b = nullptr;
  if (g == 0) {
    b = &keys.relin;
  } else {
    auto it = keys.galois.find(g);
    if (it == keys.galois.end()) throw Error(CKKS_ERR_MISSING_KEY, "missing Galois key");
    b = it->second.get();
  }
  if (!keys.compressed) return b->u64();
  const size_t N = c.N, rows = (size_t)c.n_qp, beta = (size_t)c.beta_max;
  tmp = DevBuf(&c, beta * 2 * rows * N * 8);
  CK_CUDA(cudaMemcpy2DAsync(tmp.p, 2 * rows * N * 8, b->p, rows * N * 8, rows * N * 8, beta,
                            cudaMemcpyDeviceToDevice, c.stream));
  sample_uniform_seq(c, keys.a_seed, (1ull << 40) | (g << 8), beta, c.n_qp, c.iota(),
                     tmp.u64() + rows * N, 2 * rows);
  return tmp.u64();
}

void keys_compress(Ctx& c, ckks_keys& keys) {
  if (keys.compressed) return;
  if (!keys.own_a_seed)
    throw Error(CKKS_ERR_INVALID_ARG,
                "keys drew their uniform halves from the secret's seed; generate them with a "
                "public seed to compress them");
  const size_t N = c.N, rows = (size_t)c.n_qp, beta = (size_t)c.beta_max;
  auto halve = [&](DevBuf& full) {
    DevBuf b(&c, beta * rows * N * 8);
    CK_CUDA(cudaMemcpy2DAsync(b.p, rows * N * 8, full.p, 2 * rows * N * 8, rows * N * 8, beta,
                              cudaMemcpyDeviceToDevice, c.stream));
    full = std::move(b);
  };
  halve(keys.relin);
  for (auto& kv : keys.galois) halve(*kv.second);
  keys.compressed = true;
  CK_CUDA(cudaStreamSynchronize(c.stream));
}

Ct encrypt(Ctx& c, const ckks_keys& keys, const double* values, size_t B, size_t n, int level,
           uint64_t seed, uint64_t first_index) {
  if (n > c.N / 2) throw Error(CKKS_ERR_INVALID_ARG, "more values than slots");
  if (level < 0 || level > c.L) throw Error(CKKS_ERR_LEVEL, "level out of range");
  const int l = level + 1;
  const size_t N = c.N;
  DevBuf v(&c, std::max<size_t>(B * n, 1) * 8);
  if (B * n) CK_CUDA(cudaMemcpyAsync(v.p, values, B * n * 8, cudaMemcpyHostToDevice, c.stream));
  DevBuf m(&c, B * l * N * 8);
  const int rc = encode(c, static_cast<const double*>(v.p), B, n, level, c.delta[level], m.u64());
  if (rc != CKKS_OK) throw Error(rc, "value does not fit the scale");
  std::vector<uint64_t> ids(B);
  for (size_t b = 0; b < B; b++) ids[b] = first_index + b;
  DevBuf d_ids(&c, B * 8);
  CK_CUDA(cudaMemcpyAsync(d_ids.p, ids.data(), B * 8, cudaMemcpyHostToDevice, c.stream));
  DevBuf e(&c, B * N * 8), er(&c, B * l * N * 8), a(&c, B * l * N * 8);
  sample_cbd(c, seed, d_ids.u64(), B, static_cast<int64_t*>(e.p));
  k_int_to_rns(c, static_cast<int64_t*>(e.p), er.u64(), B, l, c.iota());
  ntt_forward(c, er.u64(), B * l, c.iota(), l);
  sample_uniform(c, seed, d_ids.u64(), B, l, c.iota(), a.u64());
  Ct ct = ct_alloc(c, B, level, c.delta[level]);
  {
  Launch L_(c, K_CRYPT, 6.0 * B * l * N * 8);
  encrypt_kernel<<<grid_for(B * l * N), TPB, 0, c.stream>>>(ct->d.u64(), m.u64(), a.u64(),
                                                             er.u64(), keys.s.u64(), B, l, c.log_n,
                                                             c.dmod());
  CK_CUDA(cudaGetLastError());
  }
  CK_CUDA(cudaStreamSynchronize(c.stream));  // host ids vector goes out of scope
  return ct;
}

void decrypt(Ctx& c, const ckks_keys& keys, const ckks_ct& ct, double* out, size_t n) {
  if (n > c.N / 2) throw Error(CKKS_ERR_INVALID_ARG, "more values than slots");
  const size_t N = c.N;
  DevBuf x(&c, ct.B * N * 8);
  {
  Launch L_(c, K_CRYPT, 4.0 * ct.B * N * 8);
  decrypt_limb0_kernel<<<grid_for(ct.B * N), TPB, 0, c.stream>>>(
      ct.d.u64(), keys.s.u64(), x.u64(), ct.B, ct.level + 1, c.log_n, c.dmod());
  CK_CUDA(cudaGetLastError());
  }
  ntt_inverse(c, x.u64(), ct.B, c.iota(), 1);
  DevBuf o(&c, std::max<size_t>(ct.B * n, 1) * 8);
  if (n) decode_limb0(c, x.u64(), ct.B, ct.scale, static_cast<double*>(o.p), n);
  if (n) CK_CUDA(cudaMemcpyAsync(out, o.p, ct.B * n * 8, cudaMemcpyDeviceToHost, c.stream));
  CK_CUDA(cudaStreamSynchronize(c.stream));
}

}  // namespace ck
