/*
 * ORACLE — test infrastructure only.
 *
 * A plain, slow, obviously-correct CPU implementation of the RNS-CKKS
 * arithmetic that encrypted KAN inference runs on (the paper's "HE" section,
 * Eqs. 6-10: homomorphic add, subtract, multiply by ciphertext and by
 * plaintext, and slot rotation; the scheme is RNS-CKKS, which the paper cites
 * and does not spell out, so every internal choice below is a stated reading).
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may load this file. The GPU library shares no code, header, table or
 * constant generator with it: it re-derives every parameter on its own and
 * the tests compare the two.
 *
 * Arithmetic style: every modular product is the definition
 * ((unsigned __int128)a * b) % q; no Montgomery, Barrett or Shoup tricks.
 *
 * Pins (tests/test_oracle_*.py): schoolbook negacyclic product vs NTT
 * product, O(N^2) evaluation-definition NTT vs the fast one, NTT/iNTT
 * identity, coefficient automorphism vs NTT-domain permutation, big-integer
 * basis-conversion bounds, RFC 8439 ChaCha20 vectors, encode/decode against
 * the O(N^2) canonical-embedding sum, decrypt(op) vs plaintext op.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;
typedef __int128 i128;

#define OR_OK 0
#define OR_ERR_ARG -1
#define OR_ERR_OVERFLOW -2
#define OR_ERR_PRIME -3

/* ------------------------------------------------------------------ */
/* Scalar modular arithmetic (definitions, q < 2^62)                   */
/* ------------------------------------------------------------------ */
static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) {
  return (uint64_t)(((u128)a * b) % q);
}
static uint64_t addmod(uint64_t a, uint64_t b, uint64_t q) {
  uint64_t s = a + b;
  return s >= q ? s - q : s;
}
static uint64_t submod(uint64_t a, uint64_t b, uint64_t q) {
  return a >= b ? a - b : a + (q - b);
}
static uint64_t powmod(uint64_t b, uint64_t e, uint64_t q) {
  uint64_t r = 1 % q;
  b %= q;
  while (e) {
    if (e & 1) r = mulmod(r, b, q);
    b = mulmod(b, b, q);
    e >>= 1;
  }
  return r;
}
/* q prime: Fermat inverse. */
static uint64_t invmod(uint64_t a, uint64_t q) { return powmod(a % q, q - 2, q); }

/* signed 64-bit value -> residue mod q */
static uint64_t smod(int64_t v, uint64_t q) {
  if (v >= 0) return (uint64_t)v % q;
  uint64_t m = (uint64_t)(-(v + 1)) + 1; /* |v| without overflow */
  m %= q;
  return m ? q - m : 0;
}

uint64_t or_mulmod(uint64_t a, uint64_t b, uint64_t q) { return mulmod(a, b, q); }
uint64_t or_powmod(uint64_t b, uint64_t e, uint64_t q) { return powmod(b, e, q); }

/* Deterministic Miller-Rabin for 64-bit n (bases = first 12 primes). */
int or_is_prime(uint64_t n) {
  static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return 0;
  for (int i = 0; i < 12; i++) {
    if (n == bases[i]) return 1;
    if (n % bases[i] == 0) return 0;
  }
  uint64_t d = n - 1;
  int r = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    r++;
  }
  for (int i = 0; i < 12; i++) {
    uint64_t x = powmod(bases[i], d, n);
    if (x == 1 || x == n - 1) continue;
    int comp = 1;
    for (int k = 1; k < r; k++) {
      x = mulmod(x, x, n);
      if (x == n - 1) {
        comp = 0;
        break;
      }
    }
    if (comp) return 0;
  }
  return 1;
}

/* bit reversal of the low `bits` bits */
static uint32_t brv(uint32_t x, int bits) {
  uint32_t r = 0;
  for (int i = 0; i < bits; i++) {
    r = (r << 1) | (x & 1);
    x >>= 1;
  }
  return r;
}

/* ------------------------------------------------------------------ */
/* Parameter chain                                                      */
/* ------------------------------------------------------------------ */
/*
 * Prime chain (reading of "36 levels, scale 2^40" / "one 60-bit prime + 18
 * 40-bit primes, one 60-bit special prime"):
 *  - q0: the largest prime < 2^q0_bits with q0 = 1 mod 2N;
 *  - special primes p_0 > p_1 > ...: the next primes = 1 mod 2N below
 *    2^p_bits (skipping q0);
 *  - scale primes, top level first: Delta_L = 2^scale_bits and, for
 *    l = L..1, q_l is the prime = 1 mod 2N nearest to Delta_l^2 / 2^scale_bits
 *    (candidates c, c+2N, c-2N, c+4N, ...), then
 *    Delta_{l-1} = Delta_l * Delta_l / q_l.
 *  Every ciphertext at level l carries scale Delta_l, so a product of two
 *  level-l ciphertexts rescales exactly onto Delta_{l-1} and the per-level
 *  scales stay within one prime gap of 2^scale_bits.
 */
static int used(uint64_t c, const uint64_t* a, int na, const uint64_t* b, int nb) {
  for (int i = 0; i < na; i++)
    if (a[i] == c) return 1;
  for (int i = 0; i < nb; i++)
    if (b[i] == c) return 1;
  return 0;
}

int or_gen_chain(int log_n, int q0_bits, int scale_bits, int n_scale, int p_bits,
                 int n_special, uint64_t* q, uint64_t* p, double* delta) {
  if (log_n < 2 || log_n > 17 || q0_bits > 61 || p_bits > 61 || scale_bits > 60 ||
      scale_bits < 20 || n_scale < 0 || n_special < 1)
    return OR_ERR_ARG;
  const uint64_t M = 2ull << log_n;
  /* q0 */
  uint64_t x = (((1ull << q0_bits) - 2) / M) * M + 1;
  while (!or_is_prime(x)) x -= M;
  q[0] = x;
  /* special primes */
  x = (((1ull << p_bits) - 2) / M) * M + 1;
  for (int k = 0; k < n_special; k++) {
    while (!or_is_prime(x) || x == q[0]) x -= M;
    p[k] = x;
    x -= M;
  }
  /* scale primes, top-down */
  double d = ldexp(1.0, scale_bits);
  delta[n_scale] = d;
  for (int l = n_scale; l >= 1; l--) {
    double T = ldexp(d * d, -scale_bits);
    uint64_t k = (uint64_t)floor((T - 1.0) / (double)M + 0.5);
    uint64_t base = k * M + 1;
    uint64_t chosen = 0;
    for (int64_t off = 0; off < 100000; off++) {
      /* offsets 0, +1, -1, +2, -2, ... (in units of M) */
      int64_t s = (off + 1) / 2;
      if ((off & 1) == 0) s = -s;
      uint64_t c = base + (uint64_t)(s * (int64_t)M);
      if (or_is_prime(c) && !used(c, q, 1, p, n_special) &&
          !used(c, q + l + 1, n_scale - l, NULL, 0)) {
        chosen = c;
        break;
      }
    }
    if (!chosen) return OR_ERR_PRIME;
    q[l] = chosen;
    d = (d * d) / (double)chosen;
    delta[l - 1] = d;
  }
  return OR_OK;
}

/* psi: the first x^((q-1)/2N), x = 2,3,..., whose N-th power is -1 */
uint64_t or_find_psi(uint64_t q, int log_n) {
  const uint64_t N = 1ull << log_n, M = 2 * N;
  for (uint64_t x = 2; x < 1000000; x++) {
    uint64_t c = powmod(x, (q - 1) / M, q);
    if (powmod(c, N, q) == q - 1) return c;
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* NTT                                                                  */
/* ------------------------------------------------------------------ */
/*
 * Forward negacyclic NTT, definition:
 *   A[j] = sum_i a[i] * psi^((2*brv(j)+1)*i) mod q,
 * i.e. the evaluation of a(X) at the odd powers of psi, output in
 * bit-reversed order. The O(N^2) form is or_ntt_naive; the fast form below
 * is the radix-2 Cooley-Tukey recursion with the psi-twist merged into the
 * twiddles.
 */
void or_ntt_naive(const uint64_t* a, uint64_t* out, int log_n, uint64_t q, uint64_t psi) {
  const uint32_t N = 1u << log_n;
  for (uint32_t j = 0; j < N; j++) {
    uint64_t e = 2ull * brv(j, log_n) + 1;
    uint64_t w = powmod(psi, e, q), acc = 0, wp = 1;
    for (uint32_t i = 0; i < N; i++) {
      acc = addmod(acc, mulmod(a[i], wp, q), q);
      wp = mulmod(wp, w, q);
    }
    out[j] = acc;
  }
}

void or_ntt_forward(uint64_t* a, int log_n, uint64_t q, uint64_t psi) {
  const uint32_t N = 1u << log_n;
  for (uint32_t m = 1, t = N >> 1; m < N; m <<= 1, t >>= 1) {
    for (uint32_t i = 0; i < m; i++) {
      uint64_t w = powmod(psi, brv(m + i, log_n), q);
      for (uint32_t j = 2 * i * t; j < 2 * i * t + t; j++) {
        uint64_t u = a[j], v = mulmod(a[j + t], w, q);
        a[j] = addmod(u, v, q);
        a[j + t] = submod(u, v, q);
      }
    }
  }
}

void or_ntt_inverse(uint64_t* a, int log_n, uint64_t q, uint64_t psi) {
  const uint32_t N = 1u << log_n;
  const uint64_t psi_inv = invmod(psi, q);
  for (uint32_t m = N >> 1, t = 1; m >= 1; m >>= 1, t <<= 1) {
    for (uint32_t i = 0; i < m; i++) {
      uint64_t w = powmod(psi_inv, brv(m + i, log_n), q);
      for (uint32_t j = 2 * i * t; j < 2 * i * t + t; j++) {
        uint64_t u = a[j], v = a[j + t];
        a[j] = addmod(u, v, q);
        a[j + t] = mulmod(submod(u, v, q), w, q);
      }
    }
  }
  const uint64_t n_inv = invmod(N % q, q);
  for (uint32_t j = 0; j < N; j++) a[j] = mulmod(a[j], n_inv, q);
}

/* schoolbook product in Z_q[X]/(X^N+1) */
void or_negacyclic_mul(const uint64_t* a, const uint64_t* b, uint64_t* out, int log_n,
                       uint64_t q) {
  const uint32_t N = 1u << log_n;
  for (uint32_t k = 0; k < N; k++) out[k] = 0;
  for (uint32_t i = 0; i < N; i++)
    for (uint32_t j = 0; j < N; j++) {
      uint64_t p = mulmod(a[i], b[j], q);
      uint32_t k = i + j;
      if (k < N)
        out[k] = addmod(out[k], p, q);
      else
        out[k - N] = submod(out[k - N], p, q);
    }
}

/* Galois automorphism a(X) -> a(X^g), coefficient form (g odd). */
void or_automorphism_coef(const uint64_t* a, uint64_t* out, int log_n, uint64_t g,
                          uint64_t q) {
  const uint64_t N = 1ull << log_n, M = 2 * N;
  for (uint64_t i = 0; i < N; i++) {
    uint64_t k = (i * g) % M;
    if (k < N)
      out[k] = a[i];
    else
      out[k - N] = a[i] ? q - a[i] : 0;
  }
}

/* Same map in the NTT domain: slot j holds a(psi^(2brv(j)+1)), and
 * a(X^g) there equals a at psi^(g*(2brv(j)+1)). */
void or_automorphism_ntt(const uint64_t* a, uint64_t* out, int log_n, uint64_t g) {
  const uint64_t N = 1ull << log_n, M = 2 * N;
  for (uint64_t j = 0; j < N; j++) {
    uint64_t e = 2ull * brv((uint32_t)j, log_n) + 1;
    uint64_t e2 = (g * e) % M;
    uint64_t src = brv((uint32_t)((e2 - 1) / 2), log_n);
    out[j] = a[src];
  }
}

/* ------------------------------------------------------------------ */
/* Canonical-embedding encoder (FP64)                                   */
/* ------------------------------------------------------------------ */
/*
 * Slots: n = N/2; slot j <-> zeta^(5^j mod 2N), zeta = exp(i*pi/N).
 * With w_i = m_i + i*m_{i+n}, slot j equals sum_i (w_i zeta^i) omega^(k_j i),
 * omega = zeta^4, k_j = (5^j mod 2N - 1)/4. Encoding inverts this with an
 * inverse DFT of length n (radix-2, decimation in time over a bit-reversed
 * input), untwists by zeta^-i, scales by S/n and rounds half-to-even.
 * The twiddle table is T[k] = (cos(2*pi*k/2N), sin(2*pi*k/2N)).
 * Compiled without floating-point contraction, so every butterfly rounds
 * the same way on any IEEE-754 machine.
 */
static void twiddles(int log_n, double* tr, double* ti) {
  const uint64_t M = 2ull << log_n;
  for (uint64_t k = 0; k < M; k++) {
    const double ang = (2.0 * M_PI * (double)k) / (double)M;
    tr[k] = cos(ang);
    ti[k] = sin(ang);
  }
}

static void slot_index(int log_n, uint32_t* kj) {
  const uint64_t M = 2ull << log_n, n = 1ull << (log_n - 1);
  uint64_t e = 1;
  for (uint64_t j = 0; j < n; j++) {
    kj[j] = (uint32_t)((e - 1) / 4);
    e = (e * 5) % M;
  }
}

/* radix-2 DIT on bit-reversed input; sign = -1 for the inverse DFT */
static void dft_radix2(double* xr, double* xi, int log_n, const double* tr,
                       const double* ti, int sign) {
  const uint32_t n = 1u << (log_n - 1);
  const int lb = log_n - 1;
  for (uint32_t i = 0; i < n; i++) {
    uint32_t r = brv(i, lb);
    if (r > i) {
      double t = xr[i];
      xr[i] = xr[r];
      xr[r] = t;
      t = xi[i];
      xi[i] = xi[r];
      xi[r] = t;
    }
  }
  for (uint32_t len = 2; len <= n; len <<= 1) {
    const uint32_t half = len >> 1, step = n / len;
    for (uint32_t s = 0; s < n; s += len) {
      for (uint32_t t = 0; t < half; t++) {
        const uint32_t k = 4u * t * step;
        const double wr = tr[k];
        const double wi = sign > 0 ? ti[k] : -ti[k];
        const double br = xr[s + t + half], bi = xi[s + t + half];
        const double pr = br * wr - bi * wi;
        const double pi = br * wi + bi * wr;
        const double ar = xr[s + t], ai = xi[s + t];
        xr[s + t] = ar + pr;
        xi[s + t] = ai + pi;
        xr[s + t + half] = ar - pr;
        xi[s + t + half] = ai - pi;
      }
    }
  }
}

static int encode_slots(const double* v, const double* vi, uint64_t nv, int log_n, double scale,
                        int64_t* coeffs);

/* v: nv <= N/2 real slot values (rest zero). coeffs: N int64. */
int or_encode(const double* v, uint64_t nv, int log_n, double scale, int64_t* coeffs) {
  return encode_slots(v, NULL, nv, log_n, scale, coeffs);
}

/* complex slot values re[j] + i im[j] */
int or_encode_complex(const double* re, const double* im, uint64_t nv, int log_n, double scale,
                      int64_t* coeffs) {
  return encode_slots(re, im, nv, log_n, scale, coeffs);
}

static int encode_slots(const double* v, const double* vi, uint64_t nv, int log_n, double scale,
                        int64_t* coeffs) {
  const uint64_t n = 1ull << (log_n - 1), M = 2ull << log_n;
  if (nv > n) return OR_ERR_ARG;
  double* tr = malloc(M * sizeof(double));
  double* ti = malloc(M * sizeof(double));
  double* xr = calloc(n, sizeof(double));
  double* xi = calloc(n, sizeof(double));
  uint32_t* kj = malloc(n * sizeof(uint32_t));
  twiddles(log_n, tr, ti);
  slot_index(log_n, kj);
  for (uint64_t j = 0; j < nv; j++) {
    xr[kj[j]] = v[j];
    if (vi) xi[kj[j]] = vi[j];
  }
  dft_radix2(xr, xi, log_n, tr, ti, -1);
  const double f = scale / (double)n;
  int rc = OR_OK;
  for (uint64_t i = 0; i < n; i++) {
    const double re = xr[i] * tr[i] + xi[i] * ti[i];
    const double im = xi[i] * tr[i] - xr[i] * ti[i];
    const double a = rint(re * f), b = rint(im * f);
    if (!(fabs(a) < 9.2e18) || !(fabs(b) < 9.2e18)) {
      rc = OR_ERR_OVERFLOW;
      break;
    }
    coeffs[i] = (int64_t)a;
    coeffs[i + n] = (int64_t)b;
  }
  free(tr);
  free(ti);
  free(xr);
  free(xi);
  free(kj);
  return rc;
}

static void decode_slots(const double* m, int log_n, double* out, double* out_im, uint64_t nv);

/* m: N real coefficients already divided by the scale; out: nv slots (real parts) */
void or_decode(const double* m, int log_n, double* out, uint64_t nv) {
  decode_slots(m, log_n, out, NULL, nv);
}

/* the same with the imaginary parts */
void or_decode_complex(const double* m, int log_n, double* re, double* im, uint64_t nv) {
  decode_slots(m, log_n, re, im, nv);
}

static void decode_slots(const double* m, int log_n, double* out, double* out_im, uint64_t nv) {
  const uint64_t n = 1ull << (log_n - 1), M = 2ull << log_n;
  double* tr = malloc(M * sizeof(double));
  double* ti = malloc(M * sizeof(double));
  double* xr = malloc(n * sizeof(double));
  double* xi = malloc(n * sizeof(double));
  uint32_t* kj = malloc(n * sizeof(uint32_t));
  twiddles(log_n, tr, ti);
  slot_index(log_n, kj);
  for (uint64_t i = 0; i < n; i++) {
    const double mr = m[i], mi = m[i + n];
    xr[i] = mr * tr[i] - mi * ti[i];
    xi[i] = mr * ti[i] + mi * tr[i];
  }
  dft_radix2(xr, xi, log_n, tr, ti, +1);
  for (uint64_t j = 0; j < nv && j < n; j++) {
    out[j] = xr[kj[j]];
    if (out_im) out_im[j] = xi[kj[j]];
  }
  free(tr);
  free(ti);
  free(xr);
  free(xi);
  free(kj);
}

/* ------------------------------------------------------------------ */
/* ChaCha20 (RFC 8439) and the samplers built on it                     */
/* ------------------------------------------------------------------ */
static uint32_t rotl32(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }
#define QR(a, b, c, d)     \
  a += b;                  \
  d ^= a;                  \
  d = rotl32(d, 16);       \
  c += d;                  \
  b ^= c;                  \
  b = rotl32(b, 12);       \
  a += b;                  \
  d ^= a;                  \
  d = rotl32(d, 8);        \
  c += d;                  \
  b ^= c;                  \
  b = rotl32(b, 7);

void or_chacha20_quarter(uint32_t* s4) {
  uint32_t a = s4[0], b = s4[1], c = s4[2], d = s4[3];
  QR(a, b, c, d);
  s4[0] = a;
  s4[1] = b;
  s4[2] = c;
  s4[3] = d;
}

void or_chacha20_block(const uint32_t* key, uint32_t counter, const uint32_t* nonce,
                       uint32_t* out) {
  uint32_t s[16], x[16];
  s[0] = 0x61707865u;
  s[1] = 0x3320646eu;
  s[2] = 0x79622d32u;
  s[3] = 0x6b206574u;
  for (int i = 0; i < 8; i++) s[4 + i] = key[i];
  s[12] = counter;
  s[13] = nonce[0];
  s[14] = nonce[1];
  s[15] = nonce[2];
  memcpy(x, s, sizeof s);
  for (int r = 0; r < 10; r++) {
    QR(x[0], x[4], x[8], x[12]);
    QR(x[1], x[5], x[9], x[13]);
    QR(x[2], x[6], x[10], x[14]);
    QR(x[3], x[7], x[11], x[15]);
    QR(x[0], x[5], x[10], x[15]);
    QR(x[1], x[6], x[11], x[12]);
    QR(x[2], x[7], x[8], x[13]);
    QR(x[3], x[4], x[9], x[14]);
  }
  for (int i = 0; i < 16; i++) out[i] = x[i] + s[i];
}

/* idx-th 32-bit keystream word of the stream (seed, domain, id):
 * key = (seed lo, seed hi, 0 x 6), nonce = (domain, id lo, id hi),
 * block counter = idx / 16, word = idx % 16. */
static uint32_t cc_word32(uint64_t seed, uint32_t domain, uint64_t id, uint64_t idx) {
  uint32_t key[8] = {(uint32_t)seed, (uint32_t)(seed >> 32), 0, 0, 0, 0, 0, 0};
  uint32_t nonce[3] = {domain, (uint32_t)id, (uint32_t)(id >> 32)};
  uint32_t blk[16];
  or_chacha20_block(key, (uint32_t)(idx / 16), nonce, blk);
  return blk[idx % 16];
}
static uint64_t cc_word64(uint64_t seed, uint32_t domain, uint64_t id, uint64_t i) {
  return (uint64_t)cc_word32(seed, domain, id, 2 * i) |
         ((uint64_t)cc_word32(seed, domain, id, 2 * i + 1) << 32);
}

uint32_t or_stream_word32(uint64_t seed, uint32_t domain, uint64_t id, uint64_t idx) {
  return cc_word32(seed, domain, id, idx);
}

/* ternary secret: s_i = (w32(seed,1,0,i) mod 3) - 1 */
void or_sample_ternary(uint64_t seed, int log_n, int64_t* s) {
  const uint64_t N = 1ull << log_n;
  for (uint64_t i = 0; i < N; i++) s[i] = (int64_t)(cc_word32(seed, 1, 0, i) % 3) - 1;
}

/* centred binomial, eta = 21: popcount(w & (2^21-1)) - popcount((w>>21) & (2^21-1)) */
void or_sample_cbd(uint64_t seed, uint64_t id, int log_n, int64_t* e) {
  const uint64_t N = 1ull << log_n;
  for (uint64_t i = 0; i < N; i++) {
    uint64_t w = cc_word64(seed, 2, id, i);
    e[i] = (int64_t)__builtin_popcountll(w & 0x1FFFFFull) -
           (int64_t)__builtin_popcountll((w >> 21) & 0x1FFFFFull);
  }
}

/* uniform mod q for stream (seed, 3, (id<<8)|t): a[i] = (w64(2i+1)*2^64 + w64(2i)) mod q */
void or_sample_uniform(uint64_t seed, uint64_t id, uint32_t t, uint64_t q, int log_n,
                       uint64_t* a) {
  const uint64_t N = 1ull << log_n;
  const uint64_t sid = (id << 8) | t;
  for (uint64_t i = 0; i < N; i++) {
    u128 v = ((u128)cc_word64(seed, 3, sid, 2 * i + 1) << 64) | cc_word64(seed, 3, sid, 2 * i);
    a[i] = (uint64_t)(v % q);
  }
}

/* ------------------------------------------------------------------ */
/* Scheme context                                                       */
/* ------------------------------------------------------------------ */
typedef struct {
  int log_n, L, alpha, beta_max, n_qp;
  uint64_t N;
  uint64_t* mod;    /* n_qp moduli: q_0..q_L then p_0..p_{alpha-1} */
  uint64_t* psi;    /* per modulus */
  double* delta;    /* L+1 canonical scales */
} or_ctx;

or_ctx* or_ctx_create(int log_n, int q0_bits, int scale_bits, int n_scale, int p_bits,
                      int n_special) {
  or_ctx* c = calloc(1, sizeof(or_ctx));
  c->log_n = log_n;
  c->N = 1ull << log_n;
  c->L = n_scale;
  c->alpha = n_special;
  c->n_qp = n_scale + 1 + n_special;
  c->beta_max = (n_scale + 1 + n_special - 1) / n_special;
  c->mod = calloc(c->n_qp, sizeof(uint64_t));
  c->psi = calloc(c->n_qp, sizeof(uint64_t));
  c->delta = calloc(n_scale + 1, sizeof(double));
  if (or_gen_chain(log_n, q0_bits, scale_bits, n_scale, p_bits, n_special, c->mod,
                   c->mod + n_scale + 1, c->delta) != OR_OK) {
    free(c->mod);
    free(c->psi);
    free(c->delta);
    free(c);
    return NULL;
  }
  for (int i = 0; i < c->n_qp; i++) c->psi[i] = or_find_psi(c->mod[i], log_n);
  return c;
}

void or_ctx_destroy(or_ctx* c) {
  if (!c) return;
  free(c->mod);
  free(c->psi);
  free(c->delta);
  free(c);
}

int or_ctx_info(const or_ctx* c, uint64_t* moduli, uint64_t* psis, double* delta) {
  for (int i = 0; i < c->n_qp; i++) {
    if (moduli) moduli[i] = c->mod[i];
    if (psis) psis[i] = c->psi[i];
  }
  if (delta)
    for (int i = 0; i <= c->L; i++) delta[i] = c->delta[i];
  return c->n_qp;
}

/* limb index of special prime k inside the QP basis */
static int pidx(const or_ctx* c, int k) { return c->L + 1 + k; }

/* NTT of a signed integer polynomial into limb t */
static void int_to_ntt(const or_ctx* c, const int64_t* v, int t, uint64_t* out) {
  for (uint64_t i = 0; i < c->N; i++) out[i] = smod(v[i], c->mod[t]);
  or_ntt_forward(out, c->log_n, c->mod[t], c->psi[t]);
}

void or_ntt_limb(const or_ctx* c, uint64_t* a, int t, int inverse) {
  if (inverse)
    or_ntt_inverse(a, c->log_n, c->mod[t], c->psi[t]);
  else
    or_ntt_forward(a, c->log_n, c->mod[t], c->psi[t]);
}

/* secret key in NTT form over all n_qp limbs; also returns the ternary coefficients */
/*
 * Sparse ternary secret of Hamming weight h (a bootstrapping key set: the
 * ModRaise overflow I grows with the secret's weight): positions by a
 * partial Fisher-Yates shuffle of 0..N-1, step i swapping i with
 * i + (w mod (N - i)) for the ChaCha20 word w = word32(seed, 4, 0, 2i), the
 * sign +1 if word32(seed, 4, 0, 2i + 1) is even, else -1.
 */
void or_sample_sparse_ternary(uint64_t seed, int log_n, int h, int64_t* s) {
  const uint64_t N = 1ull << log_n;
  uint32_t* perm = malloc(N * sizeof(uint32_t));
  for (uint64_t i = 0; i < N; i++) {
    perm[i] = (uint32_t)i;
    s[i] = 0;
  }
  for (int i = 0; i < h && (uint64_t)i < N; i++) {
    const uint64_t j = (uint64_t)i + cc_word32(seed, 4, 0, 2 * (uint64_t)i) % (N - (uint64_t)i);
    const uint32_t t = perm[i];
    perm[i] = perm[j];
    perm[j] = t;
    s[perm[i]] = (cc_word32(seed, 4, 0, 2 * (uint64_t)i + 1) & 1) ? -1 : 1;
  }
  free(perm);
}

void or_keygen_secret_sparse(const or_ctx* c, uint64_t seed, int h, uint64_t* s_ntt,
                             int64_t* s_coef) {
  int64_t* s = malloc(c->N * sizeof(int64_t));
  or_sample_sparse_ternary(seed, c->log_n, h, s);
  for (int t = 0; t < c->n_qp; t++) int_to_ntt(c, s, t, s_ntt + (uint64_t)t * c->N);
  if (s_coef) memcpy(s_coef, s, c->N * sizeof(int64_t));
  free(s);
}

void or_keygen_secret(const or_ctx* c, uint64_t seed, uint64_t* s_ntt, int64_t* s_coef) {
  int64_t* s = malloc(c->N * sizeof(int64_t));
  or_sample_ternary(seed, c->log_n, s);
  for (int t = 0; t < c->n_qp; t++) int_to_ntt(c, s, t, s_ntt + (uint64_t)t * c->N);
  if (s_coef) memcpy(s_coef, s, c->N * sizeof(int64_t));
  free(s);
}

/* s' for a Galois element g (NTT domain, all limbs); g == 0 means s^2 */
void or_target_secret(const or_ctx* c, const uint64_t* s_ntt, uint64_t g, uint64_t* sp) {
  for (int t = 0; t < c->n_qp; t++) {
    const uint64_t* st = s_ntt + (uint64_t)t * c->N;
    uint64_t* o = sp + (uint64_t)t * c->N;
    if (g == 0) {
      for (uint64_t i = 0; i < c->N; i++) o[i] = mulmod(st[i], st[i], c->mod[t]);
    } else {
      or_automorphism_ntt(st, o, c->log_n, g);
    }
  }
}

/*
 * Switching key from s' to s (hybrid, digits of alpha consecutive Q primes):
 * for digit j and every QP limb t,
 *   b = -a*s + e + (t in digit j ? [P]_{q_t} * s' : 0),   a uniform.
 * Layout: key[j][0 = b, 1 = a][t][N]. Randomness: seed, object id
 * X = 2^40 | g<<8 | j (g = 0 for relinearisation).
 */
void or_keygen_switch_pub(const or_ctx* c, uint64_t seed, uint64_t a_seed,
                          const uint64_t* s_ntt, const uint64_t* sp_ntt, uint64_t g,
                          uint64_t* key);

void or_keygen_switch(const or_ctx* c, uint64_t seed, const uint64_t* s_ntt,
                      const uint64_t* sp_ntt, uint64_t g, uint64_t* key) {
  or_keygen_switch_pub(c, seed, seed, s_ntt, sp_ntt, g, key);
}

/* The same with the uniform halves a drawn from a_seed instead of seed: a
 * public seed, independent of the secret's, from which a holder of the key
 * can regenerate a (seed-compressed keys) without learning anything of s. */
void or_keygen_switch_pub(const or_ctx* c, uint64_t seed, uint64_t a_seed,
                          const uint64_t* s_ntt, const uint64_t* sp_ntt, uint64_t g,
                          uint64_t* key) {
  const uint64_t N = c->N;
  int64_t* e = malloc(N * sizeof(int64_t));
  uint64_t* et = malloc(N * sizeof(uint64_t));
  for (int j = 0; j < c->beta_max; j++) {
    const uint64_t X = (1ull << 40) | (g << 8) | (uint64_t)j;
    or_sample_cbd(seed, X, c->log_n, e);
    for (int t = 0; t < c->n_qp; t++) {
      const uint64_t q = c->mod[t];
      uint64_t* b = key + (((uint64_t)j * 2 + 0) * c->n_qp + t) * N;
      uint64_t* a = key + (((uint64_t)j * 2 + 1) * c->n_qp + t) * N;
      or_sample_uniform(a_seed, X, (uint32_t)t, q, c->log_n, a);
      int_to_ntt(c, e, t, et);
      const int in_digit = (t <= c->L) && (t / c->alpha == j);
      uint64_t Pmod = 1 % q;
      if (in_digit)
        for (int k = 0; k < c->alpha; k++) Pmod = mulmod(Pmod, c->mod[pidx(c, k)] % q, q);
      const uint64_t* st = s_ntt + (uint64_t)t * N;
      const uint64_t* spt = sp_ntt + (uint64_t)t * N;
      for (uint64_t i = 0; i < N; i++) {
        uint64_t v = submod(et[i], mulmod(a[i], st[i], q), q);
        if (in_digit) v = addmod(v, mulmod(Pmod, spt[i], q), q);
        b[i] = v;
      }
    }
  }
  free(e);
  free(et);
}

/* encode real slots into a plaintext at `level` (NTT form, level+1 limbs) */
int or_encode_plain(const or_ctx* c, const double* v, uint64_t nv, int level, double scale,
                    uint64_t* pt) {
  int64_t* m = malloc(c->N * sizeof(int64_t));
  int rc = or_encode(v, nv, c->log_n, scale, m);
  if (rc == OR_OK)
    for (int t = 0; t <= level; t++) int_to_ntt(c, m, t, pt + (uint64_t)t * c->N);
  free(m);
  return rc;
}

int or_encode_plain_complex(const or_ctx* c, const double* re, const double* im, uint64_t nv,
                            int level, double scale, uint64_t* pt) {
  int64_t* m = malloc(c->N * sizeof(int64_t));
  int rc = or_encode_complex(re, im, nv, c->log_n, scale, m);
  if (rc == OR_OK)
    for (int t = 0; t <= level; t++) int_to_ntt(c, m, t, pt + (uint64_t)t * c->N);
  free(m);
  return rc;
}

/*
 * ModRaise (bootstrapping): a ciphertext at level 0 ([2][1][N], NTT form
 * mod q0) read as the centred coefficients of each polynomial, in
 * (-q0/2, q0/2], and reduced mod q_0 .. q_level: out [2][level+1][N], NTT
 * form. It decrypts to c0 + c1 s = m + q0 I over the integers, I a small
 * integer polynomial (|I| below about the secret's Hamming weight).
 */
void or_mod_raise(const or_ctx* c, const uint64_t* ct0, int level, uint64_t* out) {
  const uint64_t N = c->N, q0 = c->mod[0];
  uint64_t* x = malloc(N * sizeof(uint64_t));
  int64_t* v = malloc(N * sizeof(int64_t));
  for (int k = 0; k < 2; k++) {
    memcpy(x, ct0 + (uint64_t)k * N, N * sizeof(uint64_t));
    or_ntt_inverse(x, c->log_n, q0, c->psi[0]);
    for (uint64_t i = 0; i < N; i++) v[i] = x[i] > q0 / 2 ? -(int64_t)(q0 - x[i]) : (int64_t)x[i];
    for (int t = 0; t <= level; t++) int_to_ntt(c, v, t, out + ((uint64_t)k * (level + 1) + t) * N);
  }
  free(x);
  free(v);
}

/*
 * Symmetric encryption at `level` with scale Delta_level:
 *   c0 = -a*s + m + e, c1 = a  (NTT form), a_t ~ U(Z_{q_t}),
 * randomness: seed, object id = index (< 2^40).
 */
int or_encrypt(const or_ctx* c, const uint64_t* s_ntt, const double* v, uint64_t nv,
               int level, uint64_t seed, uint64_t index, uint64_t* ct) {
  const uint64_t N = c->N, l = (uint64_t)level + 1;
  int64_t* m = malloc(N * sizeof(int64_t));
  int64_t* e = malloc(N * sizeof(int64_t));
  uint64_t* mt = malloc(N * sizeof(uint64_t));
  uint64_t* et = malloc(N * sizeof(uint64_t));
  int rc = or_encode(v, nv, c->log_n, c->delta[level], m);
  if (rc == OR_OK) {
    or_sample_cbd(seed, index, c->log_n, e);
    for (uint64_t t = 0; t < l; t++) {
      const uint64_t q = c->mod[t];
      uint64_t* c0 = ct + t * N;
      uint64_t* c1 = ct + (l + t) * N;
      or_sample_uniform(seed, index, (uint32_t)t, q, c->log_n, c1);
      int_to_ntt(c, m, (int)t, mt);
      int_to_ntt(c, e, (int)t, et);
      const uint64_t* st = s_ntt + t * N;
      for (uint64_t i = 0; i < N; i++)
        c0[i] = addmod(submod(mt[i], mulmod(c1[i], st[i], q), q), et[i], q);
    }
  }
  free(m);
  free(e);
  free(mt);
  free(et);
  return rc;
}

/* Decrypt with limb 0 only: valid while |scale * value + noise| < q0/2. */
void or_decrypt(const or_ctx* c, const uint64_t* s_ntt, const uint64_t* ct, int level,
                double scale, double* out, uint64_t nv) {
  const uint64_t N = c->N, l = (uint64_t)level + 1, q = c->mod[0];
  uint64_t* x = malloc(N * sizeof(uint64_t));
  double* m = malloc(N * sizeof(double));
  for (uint64_t i = 0; i < N; i++) x[i] = addmod(ct[i], mulmod(ct[l * N + i], s_ntt[i], q), q);
  or_ntt_inverse(x, c->log_n, q, c->psi[0]);
  for (uint64_t i = 0; i < N; i++) {
    int64_t v = x[i] > q / 2 ? -(int64_t)(q - x[i]) : (int64_t)x[i];
    m[i] = (double)v / scale;
  }
  or_decode(m, c->log_n, out, nv);
  free(x);
  free(m);
}

/* ------------------------------------------------------------------ */
/* Ciphertext arithmetic; polys are [poly][limb][N], `l` limbs          */
/* ------------------------------------------------------------------ */
void or_add(const or_ctx* c, const uint64_t* a, const uint64_t* b, int n_polys, int l,
            int negate_b, uint64_t* out) {
  for (int p = 0; p < n_polys; p++)
    for (int t = 0; t < l; t++) {
      const uint64_t q = c->mod[t];
      const uint64_t off = ((uint64_t)p * l + t) * c->N;
      for (uint64_t i = 0; i < c->N; i++)
        out[off + i] = negate_b ? submod(a[off + i], b[off + i], q)
                                : addmod(a[off + i], b[off + i], q);
    }
}

/* out = a * pt (per limb), pt has >= l limbs */
void or_mul_plain(const or_ctx* c, const uint64_t* a, const uint64_t* pt, int n_polys, int l,
                  uint64_t* out) {
  for (int p = 0; p < n_polys; p++)
    for (int t = 0; t < l; t++) {
      const uint64_t q = c->mod[t];
      const uint64_t off = ((uint64_t)p * l + t) * c->N;
      for (uint64_t i = 0; i < c->N; i++)
        out[off + i] = mulmod(a[off + i], pt[(uint64_t)t * c->N + i], q);
    }
}

/* out = a * k for a signed integer constant k */
void or_mul_int(const or_ctx* c, const uint64_t* a, int64_t k, int n_polys, int l,
                uint64_t* out) {
  for (int p = 0; p < n_polys; p++)
    for (int t = 0; t < l; t++) {
      const uint64_t q = c->mod[t], kk = smod(k, q);
      const uint64_t off = ((uint64_t)p * l + t) * c->N;
      for (uint64_t i = 0; i < c->N; i++) out[off + i] = mulmod(a[off + i], kk, q);
    }
}

/* poly (first poly only, l limbs) += signed integer constant k (NTT of a constant) */
void or_add_int(const or_ctx* c, uint64_t* a, int64_t k, int l) {
  for (int t = 0; t < l; t++) {
    const uint64_t q = c->mod[t], kk = smod(k, q);
    for (uint64_t i = 0; i < c->N; i++) a[(uint64_t)t * c->N + i] = addmod(a[(uint64_t)t * c->N + i], kk, q);
  }
}

/* (a0,a1) x (b0,b1) -> (a0b0, a0b1+a1b0, a1b1) */
void or_tensor(const or_ctx* c, const uint64_t* a, const uint64_t* b, int l, uint64_t* out) {
  const uint64_t N = c->N, L = (uint64_t)l;
  for (uint64_t t = 0; t < L; t++) {
    const uint64_t q = c->mod[t];
    for (uint64_t i = 0; i < N; i++) {
      uint64_t a0 = a[t * N + i], a1 = a[(L + t) * N + i];
      uint64_t b0 = b[t * N + i], b1 = b[(L + t) * N + i];
      out[t * N + i] = mulmod(a0, b0, q);
      out[(L + t) * N + i] = addmod(mulmod(a0, b1, q), mulmod(a1, b0, q), q);
      out[(2 * L + t) * N + i] = mulmod(a1, b1, q);
    }
  }
}

void or_automorphism_polys(const or_ctx* c, const uint64_t* a, int n_rows, uint64_t g,
                           uint64_t* out) {
  for (int r = 0; r < n_rows; r++)
    or_automorphism_ntt(a + (uint64_t)r * c->N, out + (uint64_t)r * c->N, c->log_n, g);
}

/*
 * Rescale by the top prime q_l (level l -> l-1), per poly:
 *   r = centred [c]_{q_l} in (-q_l/2, q_l/2],
 *   c_i <- (c_i - r) * q_l^{-1} mod q_i for i < l.
 */
void or_rescale(const or_ctx* c, const uint64_t* in, int n_polys, int level, uint64_t* out) {
  const uint64_t N = c->N, l = (uint64_t)level + 1;
  const uint64_t ql = c->mod[level];
  uint64_t* x = malloc(N * sizeof(uint64_t));
  uint64_t* r = malloc(N * sizeof(uint64_t));
  for (int p = 0; p < n_polys; p++) {
    memcpy(x, in + ((uint64_t)p * l + level) * N, N * sizeof(uint64_t));
    or_ntt_inverse(x, c->log_n, ql, c->psi[level]);
    for (uint64_t t = 0; t < (uint64_t)level; t++) {
      const uint64_t q = c->mod[t];
      for (uint64_t i = 0; i < N; i++) {
        int64_t v = x[i] > ql / 2 ? -(int64_t)(ql - x[i]) : (int64_t)x[i];
        r[i] = smod(v, q);
      }
      or_ntt_forward(r, c->log_n, q, c->psi[t]);
      const uint64_t inv = invmod(ql % q, q);
      const uint64_t* ci = in + ((uint64_t)p * l + t) * N;
      uint64_t* o = out + ((uint64_t)p * (l - 1) + t) * N;
      for (uint64_t i = 0; i < N; i++) o[i] = mulmod(submod(ci[i], r[i], q), inv, q);
    }
  }
  free(x);
  free(r);
}

/*
 * ModUp of one polynomial d (NTT form, level `level`), all digits.
 * Output ext[j][t][N] over the QP_l basis rows t = 0..l-1 (Q limbs) then
 * l..l+alpha-1 (special primes), NTT form. For digit j with primes D_j
 * (Q limbs [j*alpha, min((j+1)*alpha, l))):
 *   rows t in D_j copy d_t;
 *   other rows: sum_{i in D_j} [x_i * Dhat_i^{-1}]_{q_i} * (Dhat_i mod m_t) mod m_t,
 *   with x_i the coefficient form of d_i and Dhat_i = prod_{k in D_j, k != i} q_k
 *   (fast basis conversion, uncentred representatives).
 */
void or_modup(const or_ctx* c, const uint64_t* d, int level, uint64_t* ext) {
  const uint64_t N = c->N;
  const int l = level + 1, rows = l + c->alpha;
  const int beta = (l + c->alpha - 1) / c->alpha;
  uint64_t* xc = malloc((uint64_t)l * N * sizeof(uint64_t));
  memcpy(xc, d, (uint64_t)l * N * sizeof(uint64_t));
  for (int t = 0; t < l; t++) or_ntt_inverse(xc + (uint64_t)t * N, c->log_n, c->mod[t], c->psi[t]);
  uint64_t* v = malloc((uint64_t)c->alpha * N * sizeof(uint64_t));
  for (int j = 0; j < beta; j++) {
    const int lo = j * c->alpha, hi = (j + 1) * c->alpha < l ? (j + 1) * c->alpha : l;
    /* v_i = x_i * Dhat_i^{-1} mod q_i */
    for (int i = lo; i < hi; i++) {
      const uint64_t qi = c->mod[i];
      uint64_t dh = 1;
      for (int k = lo; k < hi; k++)
        if (k != i) dh = mulmod(dh, c->mod[k] % qi, qi);
      const uint64_t dhi = invmod(dh, qi);
      for (uint64_t n = 0; n < N; n++) v[(uint64_t)(i - lo) * N + n] = mulmod(xc[(uint64_t)i * N + n], dhi, qi);
    }
    for (int r = 0; r < rows; r++) {
      const int t = r < l ? r : pidx(c, r - l);
      uint64_t* o = ext + ((uint64_t)j * rows + r) * N;
      if (r >= lo && r < hi) {
        memcpy(o, d + (uint64_t)r * N, N * sizeof(uint64_t));
        continue;
      }
      const uint64_t m = c->mod[t];
      for (uint64_t n = 0; n < N; n++) {
        uint64_t acc = 0;
        for (int i = lo; i < hi; i++) {
          uint64_t dh = 1;
          for (int k = lo; k < hi; k++)
            if (k != i) dh = mulmod(dh, c->mod[k] % m, m);
          acc = addmod(acc, mulmod(v[(uint64_t)(i - lo) * N + n] % m, dh, m), m);
        }
        o[n] = acc;
      }
      or_ntt_forward(o, c->log_n, m, c->psi[t]);
    }
  }
  free(xc);
  free(v);
}

/* acc_k[t] = sum_j ext[j][t] * key[j][k][t] over QP_l (k = 0, 1); ext rows
 * follow or_modup, mapped first by X -> X^g when g != 0. acc: [2][rows][N] */
static uint64_t* key_product(const or_ctx* c, const uint64_t* ext_in, int level,
                             const uint64_t* key, uint64_t g) {
  const uint64_t N = c->N;
  const int l = level + 1, rows = l + c->alpha;
  const int beta = (l + c->alpha - 1) / c->alpha;
  uint64_t* ext = malloc((uint64_t)beta * rows * N * sizeof(uint64_t));
  if (g != 0)
    or_automorphism_polys(c, ext_in, beta * rows, g, ext);
  else
    memcpy(ext, ext_in, (uint64_t)beta * rows * N * sizeof(uint64_t));
  uint64_t* acc = calloc((uint64_t)2 * rows * N, sizeof(uint64_t));
  for (int k = 0; k < 2; k++)
    for (int r = 0; r < rows; r++) {
      const int t = r < l ? r : pidx(c, r - l);
      const uint64_t m = c->mod[t];
      uint64_t* a = acc + ((uint64_t)k * rows + r) * N;
      for (int j = 0; j < beta; j++) {
        const uint64_t* e = ext + ((uint64_t)j * rows + r) * N;
        const uint64_t* kk = key + (((uint64_t)j * 2 + k) * c->n_qp + t) * N;
        for (uint64_t n = 0; n < N; n++) a[n] = addmod(a[n], mulmod(e[n], kk[n], m), m);
      }
    }
  free(ext);
  return acc;
}

/*
 * Relinearisation and rescale as one division (HMult, Eq. 8). With d0, d1
 * of the tensor product at level l (NTT form, [2][l+1][N]) and the key
 * inner product acc_k over QP_l of d2's ModUp (relinearisation key), per k:
 *   y = P d_k + acc_k over QP_l (on the special primes y = acc_k),
 *   M = P q_l, D = {q_l, p_0 .. p_{alpha-1}} (the limbs dropped),
 *   out_k[i] = (y_i - Conv_{D->Q}([y]_D)_i) * M^{-1} mod q_i, i < l,
 *   Conv_{D->Q}(y)_i = sum_{m in D} v_m ((M/m) mod q_i) - u (M mod q_i),
 *   v_m = [y_m (M/m)^{-1}]_m, u = floor(sum_m v_m / m + 1/2) in double
 * precision (m in the order q_l, p_0, ..): the conversion of the centred
 * representative of [y]_M, so out = y / M rounded to nearest. out: [2][l][N].
 * This replaces ModDown by P followed by rescaling by q_l; the result
 * differs from that sequence only in the rounding of the division.
 */
static void div_p_ql(const or_ctx* c, const uint64_t* d01, const uint64_t* acc, int level,
                     uint64_t* out);

void or_relin_rescale(const or_ctx* c, const uint64_t* d01, const uint64_t* ext_in, int level,
                      const uint64_t* key, uint64_t* out) {
  uint64_t* acc = key_product(c, ext_in, level, key, 0);
  div_p_ql(c, d01, acc, level, out);
  free(acc);
}

/*
 * The division of or_relin_rescale on its own: y = P d_k + acc_k over QP_l
 * (d01 may be NULL: y = acc_k), out_k = round(y / (P q_l)) over Q_{l-1} by
 * the centred conversion of the dropped limbs. acc: [2][l + alpha][N] (Q
 * rows, then the special primes), NTT form; out: [2][level][N].
 */
void or_div_p_ql(const or_ctx* c, const uint64_t* d01, const uint64_t* acc, int level,
                 uint64_t* out) {
  div_p_ql(c, d01, acc, level, out);
}

/* the key inner product of or_keyswitch_ext without ModDown: acc_k over
 * QP_l ([2][l + alpha][N], NTT form), the rows mapped by X -> X^g first
 * when g != 0 */
void or_key_product(const or_ctx* c, const uint64_t* ext_in, int level, const uint64_t* key,
                    uint64_t g, uint64_t* acc_out) {
  const int rows = level + 1 + c->alpha;
  uint64_t* acc = key_product(c, ext_in, level, key, g);
  memcpy(acc_out, acc, (uint64_t)2 * rows * c->N * sizeof(uint64_t));
  free(acc);
}

static void div_p_ql(const or_ctx* c, const uint64_t* d01, const uint64_t* acc, int level,
                     uint64_t* out) {
  const uint64_t N = c->N;
  const int l = level + 1, rows = l + c->alpha, A = c->alpha;
  /* the dropped moduli: D[0] = q_level, D[1 + a] = p_a */
  uint64_t* Dm = malloc((uint64_t)(A + 1) * sizeof(uint64_t));
  int* Dt = malloc((uint64_t)(A + 1) * sizeof(int));
  Dt[0] = level;
  for (int a = 0; a < A; a++) Dt[1 + a] = pidx(c, a);
  for (int m = 0; m <= A; m++) Dm[m] = c->mod[Dt[m]];
  uint64_t* y = malloc((uint64_t)(A + 1) * N * sizeof(uint64_t));
  uint64_t* conv = malloc(N * sizeof(uint64_t));
  uint64_t* uo = malloc(N * sizeof(uint64_t));
  for (int k = 0; k < 2; k++) {
    for (int m = 0; m <= A; m++) {
      const uint64_t qm = Dm[m];
      uint64_t* ym = y + (uint64_t)m * N;
      const uint64_t* am = acc + ((uint64_t)k * rows + (m == 0 ? level : l + m - 1)) * N;
      if (m == 0 && d01) { /* y = P d_k + acc_k on q_level */
        uint64_t P = 1;
        for (int a = 0; a < A; a++) P = mulmod(P, c->mod[pidx(c, a)] % qm, qm);
        const uint64_t* dk = d01 + ((uint64_t)k * l + level) * N;
        for (uint64_t n = 0; n < N; n++) ym[n] = addmod(mulmod(P, dk[n], qm), am[n], qm);
      } else {
        memcpy(ym, am, N * sizeof(uint64_t));
      }
      or_ntt_inverse(ym, c->log_n, qm, c->psi[Dt[m]]);
      uint64_t h = 1; /* (M / D[m]) mod D[m] */
      for (int o = 0; o <= A; o++)
        if (o != m) h = mulmod(h, Dm[o] % qm, qm);
      const uint64_t hi = invmod(h, qm);
      for (uint64_t n = 0; n < N; n++) ym[n] = mulmod(ym[n], hi, qm);
    }
    for (uint64_t n = 0; n < N; n++) {
      double sf = 0.0;
      for (int m = 0; m <= A; m++) sf += (double)y[(uint64_t)m * N + n] * (1.0 / (double)Dm[m]);
      uo[n] = (uint64_t)floor(sf + 0.5);
    }
    for (int i = 0; i < level; i++) {
      const uint64_t q = c->mod[i];
      uint64_t M = 1, P = 1;
      for (int m = 0; m <= A; m++) M = mulmod(M, Dm[m] % q, q);
      for (int a = 0; a < A; a++) P = mulmod(P, c->mod[pidx(c, a)] % q, q);
      for (uint64_t n = 0; n < N; n++) {
        uint64_t s = 0;
        for (int m = 0; m <= A; m++) {
          uint64_t h = 1;
          for (int o = 0; o <= A; o++)
            if (o != m) h = mulmod(h, Dm[o] % q, q);
          s = addmod(s, mulmod(y[(uint64_t)m * N + n] % q, h, q), q);
        }
        conv[n] = submod(s, mulmod(uo[n] % q, M, q), q);
      }
      or_ntt_forward(conv, c->log_n, q, c->psi[i]);
      const uint64_t Minv = invmod(M, q);
      const uint64_t* ai = acc + ((uint64_t)k * rows + i) * N;
      const uint64_t* di = d01 ? d01 + ((uint64_t)k * l + i) * N : NULL;
      uint64_t* o = out + ((uint64_t)k * level + i) * N;
      for (uint64_t n = 0; n < N; n++) {
        const uint64_t yi = di ? addmod(mulmod(P, di[n], q), ai[n], q) : ai[n];
        o[n] = mulmod(submod(yi, conv[n], q), Minv, q);
      }
    }
  }
  free(Dm);
  free(Dt);
  free(y);
  free(conv);
  free(uo);
}

/*
 * Key inner product + ModDown:
 *   acc_k[t] = sum_j ext[j][t] * key[j][k][t]   (k = 0,1; over QP_l)
 *   out_k[i] = (acc_k[i] - Conv_{P->Q}([acc_k]_P)_i) * P^{-1} mod q_i,
 *   Conv_{P->Q}(y)_i = sum_k v_k (Phat_k mod q_i) - u (P mod q_i),
 *   v_k = [y_k * Phat_k^{-1}]_{p_k}, u = floor(sum_k v_k / p_k + 1/2)
 * (the sum in double precision, k ascending): the conversion of the centred
 * representative of [acc_k]_P (Halevi, Polyakov and Shoup 2019), so out is
 * acc_k / P rounded to nearest, without the bias of the uncentred sum.
 * `ext` rows follow or_modup; if g != 0 every ext row is first mapped by the
 * NTT-domain automorphism X -> X^g (hoisted rotation: automorphism after
 * ModUp). out: [2][l][N].
 */
void or_keyswitch_ext(const or_ctx* c, const uint64_t* ext_in, int level, const uint64_t* key,
                      uint64_t g, uint64_t* out) {
  const uint64_t N = c->N;
  const int l = level + 1, rows = l + c->alpha, A = c->alpha;
  uint64_t* acc = key_product(c, ext_in, level, key, g);
  /* ModDown */
  uint64_t* y = malloc((uint64_t)A * N * sizeof(uint64_t));
  uint64_t* conv = malloc(N * sizeof(uint64_t));
  uint64_t* u = malloc(N * sizeof(uint64_t));
  for (int k = 0; k < 2; k++) {
    for (int a = 0; a < A; a++) {
      const int t = pidx(c, a);
      const uint64_t pa = c->mod[t];
      uint64_t* ya = y + (uint64_t)a * N;
      memcpy(ya, acc + ((uint64_t)k * rows + l + a) * N, N * sizeof(uint64_t));
      or_ntt_inverse(ya, c->log_n, pa, c->psi[t]);
      uint64_t ph = 1;
      for (int b = 0; b < A; b++)
        if (b != a) ph = mulmod(ph, c->mod[pidx(c, b)] % pa, pa);
      const uint64_t phi = invmod(ph, pa);
      for (uint64_t n = 0; n < N; n++) ya[n] = mulmod(ya[n], phi, pa);
    }
    for (uint64_t n = 0; n < N; n++) {
      double sf = 0.0;
      for (int a = 0; a < A; a++) sf += (double)y[(uint64_t)a * N + n] * (1.0 / (double)c->mod[pidx(c, a)]);
      u[n] = (uint64_t)floor(sf + 0.5);
    }
    for (int i = 0; i < l; i++) {
      const uint64_t q = c->mod[i];
      uint64_t P = 1;
      for (int a = 0; a < A; a++) P = mulmod(P, c->mod[pidx(c, a)] % q, q);
      for (uint64_t n = 0; n < N; n++) {
        uint64_t s = 0;
        for (int a = 0; a < A; a++) {
          uint64_t ph = 1;
          for (int b = 0; b < A; b++)
            if (b != a) ph = mulmod(ph, c->mod[pidx(c, b)] % q, q);
          s = addmod(s, mulmod(y[(uint64_t)a * N + n] % q, ph, q), q);
        }
        conv[n] = submod(s, mulmod(u[n] % q, P, q), q);
      }
      or_ntt_forward(conv, c->log_n, q, c->psi[i]);
      const uint64_t Pinv = invmod(P, q);
      const uint64_t* ai = acc + ((uint64_t)k * rows + i) * N;
      uint64_t* o = out + ((uint64_t)k * l + i) * N;
      for (uint64_t n = 0; n < N; n++) o[n] = mulmod(submod(ai[n], conv[n], q), Pinv, q);
    }
  }
  free(acc);
  free(y);
  free(conv);
  free(u);
}

/*
 * QP_l rows (the l = level + 1 Q limbs, then the alpha special primes) for
 * the double-hoisted BSGS. or_qp_mul_plain_acc: acc_k += a_k * pt row by
 * row mod the row's modulus (a, acc: [2][l + alpha][N]; pt: [l + alpha][N]).
 * or_qp_lift: out = (P sigma_g(c0) + acc0) on the Q rows, acc0 on the special
 * primes (sigma_g: X -> X^g in the NTT domain, none when g = 0; acc0 NULL is
 * zero): the first polynomial of a rotation kept in QP_l.
 */
void or_qp_mul_plain_acc(const or_ctx* c, const uint64_t* a, const uint64_t* pt, int level,
                         uint64_t* acc) {
  const uint64_t N = c->N;
  const int l = level + 1, rows = l + c->alpha;
  for (int k = 0; k < 2; k++)
    for (int r = 0; r < rows; r++) {
      const uint64_t m = c->mod[r < l ? r : pidx(c, r - l)];
      const uint64_t* ar = a + ((uint64_t)k * rows + r) * N;
      const uint64_t* pr = pt + (uint64_t)r * N;
      uint64_t* o = acc + ((uint64_t)k * rows + r) * N;
      for (uint64_t n = 0; n < N; n++) o[n] = addmod(o[n], mulmod(ar[n], pr[n], m), m);
    }
}

void or_qp_lift(const or_ctx* c, const uint64_t* c0, int level, uint64_t g, const uint64_t* acc0,
                uint64_t* out) {
  const uint64_t N = c->N;
  const int l = level + 1, rows = l + c->alpha;
  uint64_t* s = malloc((uint64_t)l * N * sizeof(uint64_t));
  if (g != 0)
    or_automorphism_polys(c, c0, l, g, s);
  else
    memcpy(s, c0, (uint64_t)l * N * sizeof(uint64_t));
  for (int r = 0; r < rows; r++) {
    uint64_t* o = out + (uint64_t)r * N;
    const uint64_t* ar = acc0 ? acc0 + (uint64_t)r * N : NULL;
    if (r >= l) {
      for (uint64_t n = 0; n < N; n++) o[n] = ar ? ar[n] : 0;
      continue;
    }
    const uint64_t q = c->mod[r];
    uint64_t P = 1;
    for (int a = 0; a < c->alpha; a++) P = mulmod(P, c->mod[pidx(c, a)] % q, q);
    for (uint64_t n = 0; n < N; n++) {
      const uint64_t v = mulmod(P, s[(uint64_t)r * N + n], q);
      o[n] = ar ? addmod(v, ar[n], q) : v;
    }
  }
  free(s);
}

uint64_t or_ext_rows(const or_ctx* c, int level) {
  const int l = level + 1;
  const int beta = (l + c->alpha - 1) / c->alpha;
  return (uint64_t)beta * (uint64_t)(l + c->alpha);
}

/* Galois element of a left rotation by `step` slots: 5^(step mod N/2) mod 2N */
uint64_t or_galois_elt(const or_ctx* c, int64_t step) {
  const int64_t n = (int64_t)(c->N / 2);
  int64_t s = ((step % n) + n) % n;
  return powmod(5, (uint64_t)s, 2 * c->N);
}
