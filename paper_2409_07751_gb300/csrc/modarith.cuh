// Device modular arithmetic on uint64 residues (q < 2^62).
//
// Products of two variable residues use Barrett reduction with the
// bit-length-dependent shift of the classical algorithm (Menezes et al.,
// Handbook of Applied Cryptography, Alg. 14.42): for x < 2^(2s),
// qhat = ((x >> (s-1)) * mu) >> (s+1), mu = floor(2^(2s)/q), and
// x - qhat*q < 3q. Products by a fixed operand w use Shoup's method with the
// precomputed w' = floor(w * 2^64 / q): a*w - hi(a*w')*q lies in [0, 2q).
#pragma once
#include <stdint.h>

#include "internal.h"

namespace ck {

__device__ __forceinline__ uint64_t add_mod(uint64_t a, uint64_t b, uint64_t q) {
  uint64_t s = a + b;
  return s >= q ? s - q : s;
}
__device__ __forceinline__ uint64_t sub_mod(uint64_t a, uint64_t b, uint64_t q) {
  return a >= b ? a - b : a + (q - b);
}
// (hi:lo) mod q for (hi:lo) < 2^(2s)
__device__ __forceinline__ uint64_t reduce128(uint64_t lo, uint64_t hi, const Mod& m) {
  const uint32_t s = m.s;
  const uint64_t x1 = (lo >> (s - 1)) | (hi << (65 - s));
  const uint64_t ql = x1 * m.mu;
  const uint64_t qh = __umul64hi(x1, m.mu);
  const uint64_t qhat = (ql >> (s + 1)) | (qh << (63 - s));
  uint64_t r = lo - qhat * m.q;
  if (r >= m.q) r -= m.q;
  if (r >= m.q) r -= m.q;
  return r;
}
// any 128-bit (hi:lo) mod q, for q of at least 33 bits
__device__ __forceinline__ uint64_t reduce_wide(uint64_t lo, uint64_t hi, const Mod& m) {
  const uint64_t h = reduce128(hi, 0, m), l = reduce128(lo, 0, m);
  const uint64_t plo = h * m.t64, phi = __umul64hi(h, m.t64);
  const uint64_t slo = plo + l;
  return reduce128(slo, phi + (slo < plo ? 1 : 0), m);
}
__device__ __forceinline__ uint64_t mul_mod(uint64_t a, uint64_t b, const Mod& m) {
  const uint64_t lo = a * b;
  const uint64_t hi = __umul64hi(a, b);
  const uint32_t s = m.s;
  const uint64_t x1 = (lo >> (s - 1)) | (hi << (65 - s));
  const uint64_t ql = x1 * m.mu;
  const uint64_t qh = __umul64hi(x1, m.mu);
  const uint64_t qhat = (ql >> (s + 1)) | (qh << (63 - s));
  uint64_t r = lo - qhat * m.q;
  if (r >= m.q) r -= m.q;
  if (r >= m.q) r -= m.q;
  return r;
}
// a w - Q q mod 2^64, formed as a w + Q (2^64 - q) in one chain of 32-bit
// pieces: the two widening low products summed, then the four cross
// products added to the high word (the remainder of every Shoup product;
// the same value as the two 64-bit products and a subtraction, measured 9 %
// faster in a butterfly)
// CHAIN = false: the same value from two 64-bit products and a subtraction
// (which of the two forms runs faster depends on the kernel's register
// pressure; the transforms choose per descriptor by measurement)
template <bool CHAIN>
__device__ __forceinline__ uint64_t mul_sub_q_t(uint64_t a, uint64_t w, uint64_t Q, uint64_t q) {
  if (!CHAIN) return a * w - Q * q;
  const uint64_t nq = 0 - q;
  const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32);
  const uint32_t Q0 = (uint32_t)Q, Q1 = (uint32_t)(Q >> 32);
  const uint32_t w0 = (uint32_t)w, w1 = (uint32_t)(w >> 32);
  const uint32_t n0 = (uint32_t)nq, n1 = (uint32_t)(nq >> 32);
  const uint64_t lo = (uint64_t)a0 * w0 + (uint64_t)Q0 * n0;
  const uint32_t hi = (uint32_t)(lo >> 32) + a0 * w1 + a1 * w0 + Q0 * n1 + Q1 * n0;
  return ((uint64_t)hi << 32) | (uint32_t)lo;
}
__device__ __forceinline__ uint64_t mul_sub_q(uint64_t a, uint64_t w, uint64_t Q, uint64_t q) {
  return mul_sub_q_t<true>(a, w, Q, q);
}
template <bool CHAIN = true>
__device__ __forceinline__ uint64_t mul_shoup_t(uint64_t a, uint64_t w, uint64_t ws, uint64_t q) {
  const uint64_t r = mul_sub_q_t<CHAIN>(a, w, __umul64hi(a, ws), q);
  return r >= q ? r - q : r;
}
__device__ __forceinline__ uint64_t mul_shoup(uint64_t a, uint64_t w, uint64_t ws, uint64_t q) {
  return mul_shoup_t<true>(a, w, ws, q);
}
// Shoup product whose quotient is estimated from three of the four 32-bit
// partial products of y * ws (the low product and the carries out of the
// middle ones are dropped): with y ws = y1 s1 2^64 + (y1 s0 + y0 s1) 2^32 +
// y0 s0, Q' = y1 s1 + hi(y1 s0) + hi(y0 s1) satisfies Q - 2 <= Q' <= Q for
// the exact Q = floor(y ws / 2^64), so y w - Q' q lies in [0, 4q) for any
// y < 2^64 (exact Shoup: [0, 2q)). The remainder by mul_sub_q.
template <bool CHAIN = true>
__device__ __forceinline__ uint64_t shoup_approx_t(uint64_t y, uint64_t w, uint64_t ws, uint64_t q) {
  const uint32_t y0 = (uint32_t)y, y1 = (uint32_t)(y >> 32);
  const uint32_t s0 = (uint32_t)ws, s1 = (uint32_t)(ws >> 32);
  const uint64_t Q = (uint64_t)y1 * s1 + __umulhi(y1, s0) + __umulhi(y0, s1);
  return mul_sub_q_t<CHAIN>(y, w, Q, q);
}
__device__ __forceinline__ uint64_t shoup_approx(uint64_t y, uint64_t w, uint64_t ws, uint64_t q) {
  return shoup_approx_t<true>(y, w, ws, q);
}
// the subtraction form (kept to measure the two forms against each other)
__device__ __forceinline__ uint64_t shoup_approx_sub(uint64_t y, uint64_t w, uint64_t ws, uint64_t q) {
  return shoup_approx_t<false>(y, w, ws, q);
}

// Forward butterfly without the reduction of x, for moduli q < 2^50: with
// t in [0, 4q) both outputs grow by less than 4q per stage, so 16 stages
// from inputs below q stay below 65q < 2^57.
template <bool CHAIN = true>
__device__ __forceinline__ void ct_grow(uint64_t& x, uint64_t& y, uint64_t w, uint64_t ws,
                                        uint64_t q, uint64_t q2) {
  const uint64_t u = x;
  const uint64_t t = shoup_approx_t<CHAIN>(y, w, ws, q);
  x = u + t;
  y = u - t + 2 * q2;
}
// x < 2^64 -> x mod q, with w1s = floor(2^64 / q) (Shoup's product by 1)
__device__ __forceinline__ uint64_t reduce_full(uint64_t x, uint64_t q, uint64_t w1s) {
  const uint64_t t = x - __umul64hi(x, w1s) * q;
  return t >= q ? t - q : t;
}
// reduction of an arbitrary 64-bit value (rarely used; plain division)
__device__ __forceinline__ uint64_t reduce64(uint64_t a, uint64_t q) { return a % q; }
// signed value -> residue (the division only runs when |v| >= q)
__device__ __forceinline__ uint64_t smod64(int64_t v, uint64_t q) {
  if (v >= 0) {
    const uint64_t u = (uint64_t)v;
    return u < q ? u : u % q;
  }
  uint64_t m = (uint64_t)(-(v + 1)) + 1;
  m = m < q ? m : m % q;
  return m ? q - m : 0;
}

// Division of a 32-bit n by a fixed divisor d >= 1 with a precomputed
// multiplier (the round-up method of Granlund and Montgomery, 1994): with
// s = ceil(log2 d) and m = floor(2^32 (2^s - d) / d) + 1,
// n / d = (hi32(n m) + n) >> s for every n < 2^32 (the sum in 64 bits).
// Kernels use it for the row -> (batch element, limb) split of their index.
struct DivU32 {
  uint32_t d, m, s;
};
inline DivU32 divu(int d) {
  DivU32 r{(uint32_t)d, 0, 0};
  while ((1ull << r.s) < r.d) r.s++;
  r.m = (uint32_t)(((1ull << 32) * ((1ull << r.s) - r.d)) / r.d + 1);
  return r;
}
__device__ __forceinline__ uint32_t udiv(uint32_t n, const DivU32& D) {
  return (uint32_t)(((uint64_t)__umulhi(n, D.m) + n) >> D.s);
}
__device__ __forceinline__ uint32_t umod(uint32_t n, const DivU32& D) {
  return n - udiv(n, D) * D.d;
}

// per-limb residues of host constants, passed by value to kernels
constexpr int MAX_LIMBS = 64;
struct LimbRes {
  uint64_t v[MAX_LIMBS];
  uint64_t s[MAX_LIMBS];  // Shoup companions floor(v 2^64 / q_t)
};

}  // namespace ck
