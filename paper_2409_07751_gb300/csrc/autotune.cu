// Key-switching digit layout chosen by measurement.
//
// Hybrid key switching splits the l Q-limbs into beta = ceil(l / alpha)
// digits and extends each to the l + alpha limbs of QP: the ModUp transforms
// and the key inner product grow with beta (l + alpha), the ModDown
// transforms with alpha, and the special modulus P (alpha primes) must not
// be smaller than the largest digit modulus for the key-switching noise to
// stay below the rescaling noise. For a given chain and a bound on log2(QP)
// (the security budget), each candidate alpha takes the largest special
// primes that fit, p_bits = min(60, floor((max_qp_bits - log2 Q) / alpha)),
// and is kept if alpha p_bits covers the largest digit (q0 and alpha - 1
// scaling primes). Each kept layout is timed on the device (HMult and HRot
// of a batch at the top level, CUDA events on the context's stream); the
// fastest wins.
#include <math.h>

#include "ops.h"

using namespace ck;

extern "C" {

int ckks_autotune_keyswitch(int log_n, int q0_bits, int scale_bits, int n_scale, int max_qp_bits,
                            int batch, int device, int* alpha, int* p_bits, int* tried,
                            double* ms, int cap, int* n_tried_out) {
  try {
    if (!alpha || !p_bits || batch < 1 || n_scale < 1) return CKKS_ERR_INVALID_ARG;
    const int log_q = q0_bits + n_scale * scale_bits;
    const int cands[] = {1, 2, 3, 4, 5, 6, 8, 10, 12};
    double best = INFINITY;
    int n_tried = 0;
    *alpha = 0;
    for (int a : cands) {
      if (a > n_scale + 1) break;
      const int p = std::min(60, (max_qp_bits - log_q) / a);
      const int digit_bits = q0_bits + (a - 1) * scale_bits;
      if (p < 30 || a * p < digit_bits) continue;
      if ((n_scale + a) / a > MAX_DIGITS) continue;  // more digits than the kernels take
      auto h = std::make_unique<ckks_ctx>();
      Ctx& c = h->c;
      ctx_init(c, log_n, q0_bits, scale_bits, n_scale, p, a, device);
      std::unique_ptr<ckks_keys> keys = keygen(c, 1, {1});
      std::vector<double> v((size_t)batch * (c.N / 2), 0.25);
      Ct x = encrypt(c, *keys, v.data(), (size_t)batch, c.N / 2, n_scale, 2, 0);
      op_mul(c, *keys, *x, *x);  // warm-up: tables of the top level
      op_rotate(c, *keys, *x, 1);
      cudaEvent_t e0, e1;
      CK_CUDA(cudaEventCreate(&e0));
      CK_CUDA(cudaEventCreate(&e1));
      CK_CUDA(cudaEventRecord(e0, c.stream));
      for (int r = 0; r < 3; r++) {
        op_mul(c, *keys, *x, *x);
        op_rotate(c, *keys, *x, 1);
      }
      CK_CUDA(cudaEventRecord(e1, c.stream));
      CK_CUDA(cudaEventSynchronize(e1));
      float t = 0;
      CK_CUDA(cudaEventElapsedTime(&t, e0, e1));
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (n_tried < cap) {
        if (ms) ms[n_tried] = t / 3.0;
        if (tried) tried[n_tried] = a;
      }
      n_tried++;
      if (t < best) {
        best = t;
        *alpha = a;
        *p_bits = p;
      }
    }
    if (n_tried_out) *n_tried_out = n_tried;
    if (*alpha == 0) throw Error(CKKS_ERR_UNSUPPORTED, "no digit layout fits the bound");
    return CKKS_OK;
  } catch (...) {
    return api_error();
  }
}

// NTT launch shape chosen by measurement: the clustered transforms run at
// two CTAs per SM (64 registers per thread, 32 warps) or one (up to 128
// registers: no spills in the fused descriptors, but half the warps). Each
// descriptor kind is a slot; the workload (HMult, HRot, a constant product,
// a rescale and a plain forward transform of a batch at the top level) runs
// with every slot at one setting, then at the other, with per-launch CUDA
// events; each slot keeps the faster. ms: [2][NTT_SLOT_COUNT] (row 0: two
// CTAs per SM, row 1: one), chosen: [NTT_SLOT_COUNT].
int ckks_autotune_ntt(ckks_ctx* ctx, int batch, double* ms, int* chosen) {
  try {
    if (!ctx || batch < 1) return CKKS_ERR_INVALID_ARG;
    Ctx& c = ctx->c;
    if (c.log_n < 15 || c.L < 2) {  // only the 2^15 and 2^16 transforms have both shapes
      for (int s = 0; s < NTT_SLOT_COUNT; s++) {
        if (chosen) chosen[s] = c.ntt_minb[s];
      }
      return CKKS_OK;
    }
    std::unique_ptr<ckks_keys> keys = keygen(c, 1, {1});
    std::vector<double> v((size_t)batch * (c.N / 2), 0.25);
    Ct x = encrypt(c, *keys, v.data(), (size_t)batch, c.N / 2, c.L, 2, 0);
    const size_t rows = (size_t)batch * 2 * (c.L + 1);
    DevBuf buf(&c, rows * c.N * 8);
    CK_CUDA(cudaMemsetAsync(buf.p, 0, buf.bytes, c.stream));
    auto work = [&]() {
      op_mul(c, *keys, *x, *x);
      op_rotate(c, *keys, *x, 1);
      op_mul_const(c, *x, 0.5);
      op_rescale(c, *x);
      ntt_forward(c, buf.u64(), rows, c.iota(), c.L + 1);
    };
    static const int slot_of_kind[][2] = {{K_NTT_FWD, NTT_SLOT_FWD}, {K_MODUP_NTT, NTT_SLOT_MODUP},
                                          {K_MODDOWN_NTT, NTT_SLOT_MODDOWN},
                                          {K_RESCALE_NTT, NTT_SLOT_RESCALE},
                                          {K_RR_NTT, NTT_SLOT_RELIN_RESCALE},
                                          {K_NTT_INV, NTT_SLOT_INV}};
    double t[2][NTT_SLOT_COUNT] = {};
    const bool prof = c.prof;
    for (int setting = 0; setting < 2; setting++) {
      for (int s = 0; s < NTT_SLOT_COUNT; s++) c.ntt_minb[s] = setting == 0 ? 2 : 1;
      work();  // warm-up (tables, attributes)
      std::vector<double> k_ms(K_KIND_COUNT, 0.0);
      CK_CUDA(cudaStreamSynchronize(c.stream));
      ckks_profile_collect2(ctx, k_ms.data(), nullptr, nullptr, nullptr, K_KIND_COUNT);
      c.prof = true;
      for (int r = 0; r < 3; r++) work();
      ckks_profile_collect2(ctx, k_ms.data(), nullptr, nullptr, nullptr, K_KIND_COUNT);
      c.prof = prof;
      for (auto& m : slot_of_kind) t[setting][m[1]] = k_ms[m[0]] / 3.0;
    }
    for (int s = 0; s < NTT_SLOT_COUNT; s++) {
      c.ntt_minb[s] = t[1][s] < t[0][s] ? 1 : 2;
      if (chosen) chosen[s] = c.ntt_minb[s];
      if (ms) {
        ms[s] = t[0][s];
        ms[NTT_SLOT_COUNT + s] = t[1][s];
      }
    }
    CK_CUDA(cudaStreamSynchronize(c.stream));
    return CKKS_OK;
  } catch (...) {
    return api_error();
  }
}

int ckks_set_ntt_shape(ckks_ctx* ctx, int slot, int ctas_per_sm) {
  if (!ctx || slot < 0 || slot >= NTT_SLOT_COUNT || (ctas_per_sm != 1 && ctas_per_sm != 2))
    return CKKS_ERR_INVALID_ARG;
  ctx->c.ntt_minb[slot] = ctas_per_sm;
  return CKKS_OK;
}

}  // extern "C"
