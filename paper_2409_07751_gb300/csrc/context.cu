// Context: parameter chain, NTT / FFT / basis-conversion tables, device memory.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "internal.h"

namespace ck {

typedef unsigned __int128 u128;

void cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return;
  if (e == cudaErrorMemoryAllocation)
    throw Error(CKKS_ERR_OUT_OF_MEMORY, std::string("out of device memory: ") + what);
  throw Error(CKKS_ERR_CUDA, std::string(cudaGetErrorString(e)) + " in " + what);
}

DevBuf::DevBuf(Ctx* c, size_t b) : ctx(c), bytes(b) {
  if (b) CK_CUDA(cudaMallocAsync(&p, b, c->stream));
}
DevBuf::~DevBuf() { reset(); }
void DevBuf::reset() {
  if (p && ctx) cudaFreeAsync(p, ctx->stream);
  p = nullptr;
  bytes = 0;
}
DevBuf& DevBuf::operator=(DevBuf&& o) noexcept {
  if (this != &o) {
    reset();
    ctx = o.ctx;
    p = o.p;
    bytes = o.bytes;
    o.p = nullptr;
    o.bytes = 0;
  }
  return *this;
}

const char* kernel_kind_name(int k) {
  static const char* names[K_KIND_COUNT] = {
      "ntt_small", "ntt_fwd", "ntt_inv", "modup_ntt", "moddown_ntt", "rescale_ntt",
      "modup", "key_inner_product", "moddown_conv", "moddown_finish", "tensor", "mul_plain",
      "add", "mul_int", "lincomb", "rotate_finish", "automorphism", "rescale_spread",
      "rescale_finish", "int_to_rns", "encode_fft", "sample", "crypt", "copy",
      "relin_rescale_ntt", "relin_rescale_top", "conversion_overflow"};
  return (k >= 0 && k < K_KIND_COUNT) ? names[k] : "?";
}

cudaEvent_t Ctx::take_event() {
  if (!ev_pool.empty()) {
    cudaEvent_t e = ev_pool.back();
    ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  CK_CUDA(cudaEventCreate(&e));
  return e;
}

Launch::Launch(Ctx& cx, int k, double algorithmic_bytes, double modmuls)
    : c(cx), kind(k), bytes(algorithmic_bytes) {
  c.launches[k]++;
  if (c.prof) {
    cudaEvent_t a = c.take_event();
    b = c.take_event();
    // inside a graph capture the records become event-record nodes
    CK_CUDA(c.prof_sink ? cudaEventRecordWithFlags(a, c.stream, cudaEventRecordExternal)
                        : cudaEventRecord(a, c.stream));
    (c.prof_sink ? *c.prof_sink : c.prof_recs).push_back(ProfRec{k, bytes, modmuls, a, b});
  }
}
Launch::~Launch() {
  if (b) {
    if (c.prof_sink)
      cudaEventRecordWithFlags(b, c.stream, cudaEventRecordExternal);
    else
      cudaEventRecord(b, c.stream);
  }
}

// ------------------------------------------------------------------ host math
uint64_t mulmod_h(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a * b) % q); }
uint64_t powmod_h(uint64_t b, uint64_t e, uint64_t q) {
  uint64_t r = 1 % q;
  b %= q;
  for (; e; e >>= 1) {
    if (e & 1) r = mulmod_h(r, b, q);
    b = mulmod_h(b, b, q);
  }
  return r;
}
uint64_t invmod_h(uint64_t a, uint64_t q) { return powmod_h(a % q, q - 2, q); }
uint64_t shoup_h(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) / q); }
Mod make_mod(uint64_t q) {
  Mod m;
  m.q = q;
  m.s = 64 - __builtin_clzll(q);
  m.mu = (uint64_t)(((u128)1 << (2 * m.s)) / q);
  m.pad = 0;
  m.t64 = (uint64_t)((((u128)1) << 64) % q);
  return m;
}

bool is_prime_h(uint64_t n) {
  const uint64_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return false;
  for (uint64_t p : small) {
    if (n == p) return true;
    if (n % p == 0) return false;
  }
  uint64_t d = n - 1;
  int r = 0;
  while (!(d & 1)) d >>= 1, r++;
  for (uint64_t a : small) {
    uint64_t x = powmod_h(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool witness = true;
    for (int i = 1; i < r && witness; i++) {
      x = mulmod_h(x, x, n);
      if (x == n - 1) witness = false;
    }
    if (witness) return false;
  }
  return true;
}

// Prime chain rule (same rule as documented in the ABI header).
int gen_chain(int log_n, int q0_bits, int scale_bits, int n_scale, int p_bits, int n_special,
              std::vector<uint64_t>& mod, std::vector<double>& delta) {
  const uint64_t M = 2ull << log_n;
  std::vector<uint64_t> q(n_scale + 1), p(n_special);
  uint64_t x = (((1ull << q0_bits) - 2) / M) * M + 1;
  while (!is_prime_h(x)) x -= M;
  q[0] = x;
  x = (((1ull << p_bits) - 2) / M) * M + 1;
  for (int k = 0; k < n_special; k++) {
    while (!is_prime_h(x) || x == q[0]) x -= M;
    p[k] = x;
    x -= M;
  }
  delta.assign(n_scale + 1, 0.0);
  double d = ldexp(1.0, scale_bits);
  delta[n_scale] = d;
  for (int l = n_scale; l >= 1; l--) {
    const double T = ldexp(d * d, -scale_bits);
    const uint64_t base = (uint64_t)floor((T - 1.0) / (double)M + 0.5) * M + 1;
    uint64_t chosen = 0;
    for (int64_t step = 0; step < 100000 && !chosen; step++) {
      int64_t k = (step + 1) / 2;
      if (!(step & 1)) k = -k;
      const uint64_t c = base + (uint64_t)(k * (int64_t)M);
      if (!is_prime_h(c)) continue;
      bool taken = (c == q[0]);
      for (uint64_t v : p) taken |= (v == c);
      for (int j = l + 1; j <= n_scale; j++) taken |= (q[j] == c);
      if (!taken) chosen = c;
    }
    if (!chosen) return CKKS_ERR_INVALID_ARG;
    q[l] = chosen;
    d = (d * d) / (double)chosen;
    delta[l - 1] = d;
  }
  mod = q;
  mod.insert(mod.end(), p.begin(), p.end());
  return CKKS_OK;
}

static uint64_t find_psi(uint64_t q, int log_n) {
  const uint64_t N = 1ull << log_n, M = 2 * N;
  for (uint64_t x = 2; x < 1000000; x++) {
    const uint64_t c = powmod_h(x, (q - 1) / M, q);
    if (powmod_h(c, N, q) == q - 1) return c;
  }
  throw Error(CKKS_ERR_INVALID_ARG, "no 2N-th root of unity");
}

static uint32_t brv_h(uint32_t x, int bits) {
  uint32_t r = 0;
  for (int i = 0; i < bits; i++) r = (r << 1) | ((x >> i) & 1);
  return r;
}

template <class T>
static DevBuf upload(Ctx* c, const std::vector<T>& v) {
  DevBuf b(c, v.size() * sizeof(T));
  if (!v.empty()) CK_CUDA(cudaMemcpyAsync(b.p, v.data(), b.bytes, cudaMemcpyHostToDevice, c->stream));
  return b;
}

void ctx_init(Ctx& c, int log_n, int q0_bits, int scale_bits, int n_scale, int p_bits,
              int n_special, int device) {
  if (log_n < 2 || log_n > 16 || q0_bits < 30 || q0_bits > 61 || p_bits < 30 || p_bits > 61 ||
      scale_bits < 20 || scale_bits > 60 || n_scale < 0 || n_scale > 60 || n_special < 1 ||
      n_special > 16)
    throw Error(CKKS_ERR_INVALID_ARG, "parameter out of range");
  c.device = device;
  CK_CUDA(cudaSetDevice(device));
  CK_CUDA(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking));
  c.own_stream = true;
  {
    cudaMemPool_t pool;
    CK_CUDA(cudaDeviceGetDefaultMemPool(&pool, device));
    uint64_t thr = UINT64_MAX;
    CK_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
  }
  c.log_n = log_n;
  c.N = 1ull << log_n;
  c.L = n_scale;
  c.alpha = n_special;
  c.n_qp = n_scale + 1 + n_special;
  c.beta_max = (n_scale + 1 + n_special - 1) / n_special;
  if (gen_chain(log_n, q0_bits, scale_bits, n_scale, p_bits, n_special, c.mod, c.delta) != CKKS_OK)
    throw Error(CKKS_ERR_INVALID_ARG, "prime chain generation failed");
  const uint64_t N = c.N;
  c.psi.resize(c.n_qp);
  std::vector<Mod> mods(c.n_qp);
  std::vector<uint64_t> tw(c.n_qp * N), tws(c.n_qp * N), itw(c.n_qp * N), itws(c.n_qp * N);
  std::vector<uint64_t> ninv(c.n_qp), ninvs(c.n_qp);
  for (int t = 0; t < c.n_qp; t++) {
    const uint64_t q = c.mod[t];
    mods[t] = make_mod(q);
    c.psi[t] = find_psi(q, log_n);
    const uint64_t pinv = invmod_h(c.psi[t], q);
    // powers psi^e for e < N, then scatter to bit-reversed index
    uint64_t w = 1, wi = 1;
    for (uint64_t e = 0; e < N; e++) {
      const uint32_t k = brv_h((uint32_t)e, log_n);
      tw[t * N + k] = w;
      itw[t * N + k] = wi;
      w = mulmod_h(w, c.psi[t], q);
      wi = mulmod_h(wi, pinv, q);
    }
    for (uint64_t k = 0; k < N; k++) {
      tws[t * N + k] = shoup_h(tw[t * N + k], q);
      itws[t * N + k] = shoup_h(itw[t * N + k], q);
    }
    ninv[t] = invmod_h(N % q, q);
    ninvs[t] = shoup_h(ninv[t], q);
  }
  if (log_n > 12) {
    // rounds with base distance s = 2^ls, ls = 9, 6, 3, 0: nodes m4 + B8,
    // m4 = N / (8 s), B8 < m4, stored consecutively round after round
    size_t nodes = 0;
    for (int ls = 9; ls >= 0; ls -= 3) nodes += N >> (ls + 3);
    c.tw8_nodes = nodes;
    std::vector<uint64_t> t8((size_t)c.n_qp * nodes * 14), it8((size_t)c.n_qp * nodes * 14);
    for (int t = 0; t < c.n_qp; t++) {
      size_t node = (size_t)t * nodes;
      for (int ls = 9; ls >= 0; ls -= 3) {
        const uint64_t m4 = N >> (ls + 3);
        for (uint64_t B8 = 0; B8 < m4; B8++, node++) {
          const uint64_t idx[7] = {m4 + B8, 2 * m4 + 2 * B8, 2 * m4 + 2 * B8 + 1, 4 * m4 + 4 * B8,
                                   4 * m4 + 4 * B8 + 1, 4 * m4 + 4 * B8 + 2, 4 * m4 + 4 * B8 + 3};
          for (int k = 0; k < 7; k++) {
            t8[node * 14 + 2 * k] = tw[t * N + idx[k]];
            t8[node * 14 + 2 * k + 1] = tws[t * N + idx[k]];
            it8[node * 14 + 2 * k] = itw[t * N + idx[k]];
            it8[node * 14 + 2 * k + 1] = itws[t * N + idx[k]];
          }
        }
      }
    }
    c.d_tw8 = upload(&c, t8);
    c.d_itw8 = upload(&c, it8);
  }
  c.d_mod = upload(&c, mods);
  c.d_tw = upload(&c, tw);
  c.d_tws = upload(&c, tws);
  c.d_itw = upload(&c, itw);
  c.d_itws = upload(&c, itws);
  c.d_ninv = upload(&c, ninv);
  c.d_ninvs = upload(&c, ninvs);
  std::vector<int16_t> iota(c.n_qp);
  for (int t = 0; t < c.n_qp; t++) iota[t] = (int16_t)t;
  c.d_iota = upload(&c, iota);
  // encoder twiddles and slot permutation
  const uint64_t M = 2 * N;
  std::vector<double> fft(2 * M);
  for (uint64_t k = 0; k < M; k++) {
    const double ang = (2.0 * M_PI * (double)k) / (double)M;
    fft[2 * k] = cos(ang);
    fft[2 * k + 1] = sin(ang);
  }
  c.d_fft = upload(&c, fft);
  std::vector<uint32_t> slot(N / 2);
  uint64_t e = 1;
  for (uint64_t j = 0; j < N / 2; j++) {
    slot[j] = (uint32_t)((e - 1) / 4);
    e = (e * 5) % M;
  }
  c.d_slot = upload(&c, slot);
  // ModDown constants (independent of the level)
  const int A = c.alpha;
  std::vector<uint64_t> yinv(A), yinvs(A), ph((size_t)A * (c.L + 1)), phs((size_t)A * (c.L + 1));
  for (int a = 0; a < A; a++) {
    const uint64_t pa = c.mod[c.L + 1 + a];
    uint64_t h = 1;
    for (int b = 0; b < A; b++)
      if (b != a) h = mulmod_h(h, c.mod[c.L + 1 + b] % pa, pa);
    yinv[a] = invmod_h(h, pa);
    yinvs[a] = shoup_h(yinv[a], pa);
    for (int i = 0; i <= c.L; i++) {
      const uint64_t q = c.mod[i];
      uint64_t hq = 1;
      for (int b = 0; b < A; b++)
        if (b != a) hq = mulmod_h(hq, c.mod[c.L + 1 + b] % q, q);
      ph[(size_t)a * (c.L + 1) + i] = hq;
      phs[(size_t)a * (c.L + 1) + i] = shoup_h(hq, q);
    }
  }
  c.d_md_yinv = upload(&c, yinv);
  c.d_md_yinv_s = upload(&c, yinvs);
  c.d_md_ph = upload(&c, ph);
  c.d_md_ph_s = upload(&c, phs);
  std::vector<uint64_t> rs((size_t)(c.L + 1) * (c.L + 1), 0), rss((size_t)(c.L + 1) * (c.L + 1), 0);
  for (int l = 1; l <= c.L; l++)
    for (int t = 0; t < l; t++) {
      rs[(size_t)l * (c.L + 1) + t] = invmod_h(c.mod[l] % c.mod[t], c.mod[t]);
      rss[(size_t)l * (c.L + 1) + t] = shoup_h(rs[(size_t)l * (c.L + 1) + t], c.mod[t]);
    }
  c.d_rs_inv = upload(&c, rs);
  c.d_rs_invs = upload(&c, rss);
  std::vector<uint64_t> pm(c.L + 1);
  for (int t = 0; t <= c.L; t++) {
    uint64_t P = 1 % c.mod[t];
    for (int a = 0; a < A; a++) P = mulmod_h(P, c.mod[c.L + 1 + a] % c.mod[t], c.mod[t]);
    pm[t] = P;
  }
  c.d_pmod = upload(&c, pm);
  c.d_flag = DevBuf(&c, 16);
  CK_CUDA(cudaMemsetAsync(c.d_flag.p, 0, 16, c.stream));
  CK_CUDA(cudaStreamSynchronize(c.stream));
}

Ctx::~Ctx() {
  if (stream) cudaStreamSynchronize(stream);
  for (auto& r : prof_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : ev_pool) cudaEventDestroy(e);
  conv.clear();
  perms.clear();
  scaled.clear();
  d_mod.reset();
  d_tw.reset();
  d_tws.reset();
  d_itw.reset();
  d_itws.reset();
  d_tw8.reset();
  d_itw8.reset();
  d_ninv.reset();
  d_ninvs.reset();
  d_iota.reset();
  d_fft.reset();
  d_slot.reset();
  d_md_yinv.reset();
  d_md_yinv_s.reset();
  d_md_ph.reset();
  d_md_ph_s.reset();
  d_flag.reset();
  d_rs_inv.reset();
  d_rs_invs.reset();
  d_pmod.reset();
  if (stream) cudaStreamSynchronize(stream);
  if (own_stream && stream) cudaStreamDestroy(stream);
}

// Basis-conversion tables for one level.
ConvTables& Ctx::tables(int level) {
  auto it = conv.find(level);
  if (it != conv.end()) return *it->second;
  auto T = std::make_unique<ConvTables>();
  const int l = level + 1, A = alpha, rows = l + A;
  const int beta = (l + A - 1) / A;
  T->l = l;
  T->beta = beta;
  T->rows = rows;
  std::vector<uint64_t> dhinv((size_t)beta * A, 0), dhinvs((size_t)beta * A, 0);
  std::vector<uint64_t> dh((size_t)beta * A * rows, 0), dhs((size_t)beta * A * rows, 0);
  std::vector<uint64_t> dhw((size_t)beta * A * rows, 0), dhws((size_t)beta * A * rows, 0);
  std::vector<int16_t> pat((size_t)beta * rows);
  auto row_mod = [&](int r) { return r < l ? r : L + 1 + (r - l); };
  for (int j = 0; j < beta; j++) {
    const int lo = j * A, hi = std::min((j + 1) * A, l);
    for (int i = lo; i < hi; i++) {
      const uint64_t qi = mod[i];
      uint64_t h = 1;
      for (int k = lo; k < hi; k++)
        if (k != i) h = mulmod_h(h, mod[k] % qi, qi);
      dhinv[(size_t)j * A + (i - lo)] = invmod_h(h, qi);
      dhinvs[(size_t)j * A + (i - lo)] = shoup_h(dhinv[(size_t)j * A + (i - lo)], qi);
      for (int r = 0; r < rows; r++) {
        const uint64_t m = mod[row_mod(r)];
        uint64_t hm = 1;
        for (int k = lo; k < hi; k++)
          if (k != i) hm = mulmod_h(hm, mod[k] % m, m);
        dh[((size_t)j * A + (i - lo)) * rows + r] = hm;
        dhs[((size_t)j * A + (i - lo)) * rows + r] = shoup_h(hm, m);
        // the forward transform's first twiddle psi^(brv 1) = psi^(N/2)
        const uint64_t hw = mulmod_h(hm, powmod_h(psi[row_mod(r)], N / 2, m), m);
        dhw[((size_t)j * A + (i - lo)) * rows + r] = hw;
        dhws[((size_t)j * A + (i - lo)) * rows + r] = shoup_h(hw, m);
      }
    }
    for (int r = 0; r < rows; r++)
      pat[(size_t)j * rows + r] = (r >= lo && r < hi) ? (int16_t)-1 : (int16_t)row_mod(r);
  }
  std::vector<int16_t> pq(rows);
  for (int r = 0; r < rows; r++) pq[r] = r < l ? (int16_t)-1 : (int16_t)row_mod(r);
  std::vector<uint64_t> pinv(l), pinvs(l);
  for (int i = 0; i < l; i++) {
    uint64_t P = 1;
    for (int a = 0; a < A; a++) P = mulmod_h(P, mod[L + 1 + a] % mod[i], mod[i]);
    pinv[i] = invmod_h(P, mod[i]);
    pinvs[i] = shoup_h(pinv[i], mod[i]);
  }
  T->dhinv = upload(this, dhinv);
  T->dhinv_s = upload(this, dhinvs);
  T->dh = upload(this, dh);
  T->dh_s = upload(this, dhs);
  T->dhw = upload(this, dhw);
  T->dhw_s = upload(this, dhws);
  T->ext_pattern = upload(this, pat);
  T->pq_pattern = upload(this, pq);
  std::vector<int16_t> qp(rows);
  for (int r = 0; r < rows; r++) qp[r] = (int16_t)row_mod(r);
  T->qp_pattern = upload(this, qp);
  T->md_pinv = upload(this, pinv);
  T->md_pinv_s = upload(this, pinvs);
  std::vector<uint64_t> xp(l), xps(l), mp(rows, 0), mps(rows, 0);
  for (int j = 0; j < beta; j++)
    for (int i = j * A; i < std::min((j + 1) * A, l); i++) {
      const uint64_t ninv = invmod_h(N % mod[i], mod[i]);
      xp[i] = mulmod_h(ninv, dhinv[(size_t)j * A + (i - j * A)], mod[i]);
      xps[i] = shoup_h(xp[i], mod[i]);
    }
  for (int a = 0; a < A; a++) {
    const uint64_t pa = mod[L + 1 + a];
    uint64_t h = 1;
    for (int b = 0; b < A; b++)
      if (b != a) h = mulmod_h(h, mod[L + 1 + b] % pa, pa);
    mp[l + a] = mulmod_h(invmod_h(N % pa, pa), invmod_h(h, pa), pa);
    mps[l + a] = shoup_h(mp[l + a], pa);
  }
  T->xs_post = upload(this, xp);
  T->xs_post_s = upload(this, xps);
  T->md_post = upload(this, mp);
  T->md_post_s = upload(this, mps);
  {
    std::vector<double> inv(A);
    for (int a = 0; a < A; a++) inv[a] = 1.0 / (double)mod[L + 1 + a];
    std::vector<uint64_t> pq(l), pqs(l);
    for (int i = 0; i < l; i++) {
      uint64_t P = 1;
      for (int a = 0; a < A; a++) P = mulmod_h(P, mod[L + 1 + a] % mod[i], mod[i]);
      pq[i] = P;
      pqs[i] = shoup_h(P, mod[i]);
    }
    T->md_inv = upload(this, inv);
    T->md_inv_h = inv;
    T->md_pq = upload(this, pq);
    T->md_pq_s = upload(this, pqs);
  }
  // merged relinearise + rescale (levels >= 1): D = {q_level, p_0 .. p_{A-1}}
  if (level >= 1) {
    std::vector<int> Dt = {level};
    for (int a = 0; a < A; a++) Dt.push_back(L + 1 + a);
    const int nD = A + 1;
    std::vector<int16_t> rp(rows, -1);
    std::vector<uint64_t> rpost(rows, 0), rposts(rows, 0), yinv(nD), yinvs(nD);
    std::vector<uint64_t> mh((size_t)nD * l, 0), mhs((size_t)nD * l, 0), minv(l), minvs(l);
    for (int m = 0; m < nD; m++) {
      const uint64_t qm = mod[Dt[m]];
      uint64_t h = 1;
      for (int o = 0; o < nD; o++)
        if (o != m) h = mulmod_h(h, mod[Dt[o]] % qm, qm);
      yinv[m] = invmod_h(h, qm);
      yinvs[m] = shoup_h(yinv[m], qm);
      const int r = level + m;  // acc rows level, l, .., l + A - 1
      rp[r] = (int16_t)Dt[m];
      rpost[r] = mulmod_h(invmod_h(N % qm, qm), yinv[m], qm);
      rposts[r] = shoup_h(rpost[r], qm);
      for (int i = 0; i < l; i++) {
        uint64_t hi = 1;
        for (int o = 0; o < nD; o++)
          if (o != m) hi = mulmod_h(hi, mod[Dt[o]] % mod[i], mod[i]);
        mh[(size_t)m * l + i] = hi;
        mhs[(size_t)m * l + i] = shoup_h(hi, mod[i]);
      }
    }
    std::vector<uint64_t> mq(l), mqs(l);
    std::vector<double> rinv(nD);
    for (int m = 0; m < nD; m++) rinv[m] = 1.0 / (double)mod[Dt[m]];
    for (int i = 0; i < l; i++) {
      uint64_t Mi = 1;
      for (int o = 0; o < nD; o++) Mi = mulmod_h(Mi, mod[Dt[o]] % mod[i], mod[i]);
      minv[i] = i == level ? 0 : invmod_h(Mi, mod[i]);
      minvs[i] = shoup_h(minv[i], mod[i]);
      mq[i] = Mi;
      mqs[i] = shoup_h(Mi, mod[i]);
    }
    T->rr_inv = upload(this, rinv);
    T->rr_inv_h = rinv;
    T->rr_mq = upload(this, mq);
    T->rr_mq_s = upload(this, mqs);
    uint64_t Pq = 1;
    for (int a = 0; a < A; a++) Pq = mulmod_h(Pq, mod[L + 1 + a] % mod[level], mod[level]);
    T->rr_pq = Pq;
    T->rr_pq_s = shoup_h(Pq, mod[level]);
    T->rr_pattern = upload(this, rp);
    T->rr_post = upload(this, rpost);
    T->rr_post_s = upload(this, rposts);
    T->rr_yinv = upload(this, yinv);
    T->rr_yinv_s = upload(this, yinvs);
    T->rr_mh = upload(this, mh);
    T->rr_mh_s = upload(this, mhs);
    T->rr_minv = upload(this, minv);
    T->rr_minv_s = upload(this, minvs);
  }
  auto& ref = *T;
  conv[level] = std::move(T);
  return ref;
}

const uint64_t* Ctx::scaled_consts(int r, int64_t k) {
  auto key = std::make_pair(r, k);
  auto it = scaled.find(key);
  if (it != scaled.end()) return it->second->u64();
  auto res = [&](uint64_t q) {  // k mod q for the signed k
    const uint64_t m = (uint64_t)(k < 0 ? -(k + 1) : k) % q;
    return k < 0 ? (q - 1 - m) % q : m;
  };
  std::vector<uint64_t> v(2 + 2 * (size_t)r);
  const uint64_t qr = mod[r];
  v[0] = mulmod_h(invmod_h(N % qr, qr), res(qr), qr);
  v[1] = shoup_h(v[0], qr);
  for (int t = 0; t < r; t++) {
    const uint64_t q = mod[t];
    v[2 + t] = mulmod_h(res(q), invmod_h(qr % q, q), q);
    v[2 + r + t] = shoup_h(v[2 + t], q);
  }
  auto b = std::make_unique<DevBuf>(upload(this, v));
  const uint64_t* p = b->u64();
  scaled[key] = std::move(b);
  return p;
}

uint64_t Ctx::galois(int64_t step) const {
  const int64_t n = (int64_t)(N / 2);
  const int64_t s = ((step % n) + n) % n;
  return powmod_h(5, (uint64_t)s, 2 * N);
}

// NTT-domain automorphism X -> X^g: slot j holds a(psi^(2brv(j)+1)); the
// image there is a at psi^(g (2brv(j)+1)).
const uint32_t* Ctx::perm(uint64_t g) {
  auto it = perms.find(g);
  if (it != perms.end()) return static_cast<const uint32_t*>(it->second->p);
  std::vector<uint32_t> p(N);
  const uint64_t M = 2 * N;
  for (uint64_t j = 0; j < N; j++) {
    const uint64_t e = 2ull * brv_h((uint32_t)j, log_n) + 1;
    const uint64_t e2 = (g * e) % M;
    p[j] = brv_h((uint32_t)((e2 - 1) / 2), log_n);
  }
  // The staged key inner product copies, for each aligned tile of T outputs
  // (T = 16 .. 256), the aligned tile of T sources: the permutation must map
  // every such tile into one tile. It does (only the low log2 T bits of the
  // index are permuted); checked here so a copy can never miss a source.
  for (int s = 4; s <= 8 && s <= log_n; s++) {
    const uint32_t mask = ~((1u << s) - 1);
    for (uint64_t j = 0; j < N; j++)
      if ((p[j] & mask) != (p[j & mask] & mask))
        throw Error(CKKS_ERR_UNSUPPORTED, "automorphism table is not tile-local");
  }
  auto b = std::make_unique<DevBuf>(upload(this, p));
  const uint32_t* r = static_cast<const uint32_t*>(b->p);
  perms[g] = std::move(b);
  return r;
}

void Ctx::check_waits() {
  unsigned w = 0;
  CK_CUDA(cudaMemcpyAsync(&w, wait_status(), 4, cudaMemcpyDeviceToHost, stream));
  CK_CUDA(cudaStreamSynchronize(stream));
  if (w) {
    CK_CUDA(cudaMemsetAsync(wait_status(), 0, 4, stream));
    throw Error(CKKS_ERR_TIMEOUT,
                "a device wait for staged copies ran past its limit; results since the last "
                "synchronize are invalid");
  }
}

}  // namespace ck
