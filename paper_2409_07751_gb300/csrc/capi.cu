// C ABI entry points (include/ckks_kan.h): argument checks, exception to
// error-code translation, handle ownership.
#include <string.h>

#include "ops.h"

using namespace ck;

namespace {
thread_local std::string g_last_error;
}  // namespace

int ck::api_error() {
  try {
    throw;
  } catch (const Error& e) {
    g_last_error = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host out of memory";
    return CKKS_ERR_OUT_OF_MEMORY;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return CKKS_ERR_CUDA;
  } catch (...) {
    g_last_error = "unknown error";
    return CKKS_ERR_CUDA;
  }
}

namespace {
template <class F>
int guard(F&& f) {
  try {
    f();
    return CKKS_OK;
  } catch (...) {
    return api_error();
  }
}

void need(bool cond, const char* what) {
  if (!cond) throw Error(CKKS_ERR_INVALID_ARG, what);
}
}  // namespace

extern "C" {

const char* ckks_strerror(int code) {
  switch (code) {
    case CKKS_OK: return "ok";
    case CKKS_ERR_INVALID_ARG: return "invalid argument";
    case CKKS_ERR_LEVEL: return "level exhausted or incompatible levels";
    case CKKS_ERR_SCALE: return "scale mismatch";
    case CKKS_ERR_MISSING_KEY: return "missing Galois key";
    case CKKS_ERR_OUT_OF_MEMORY: return "out of memory";
    case CKKS_ERR_CUDA: return "CUDA error";
    case CKKS_ERR_OVERFLOW: return "value does not fit its scale";
    case CKKS_ERR_TIMEOUT: return "timeout";
    case CKKS_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown error code";
  }
}

const char* ckks_last_error(void) { return g_last_error.c_str(); }

int ckks_context_create(int log_n, int q0_bits, int scale_bits, int n_scale, int p_bits,
                        int n_special, int device, ckks_ctx** out) {
  return guard([&] {
    need(out != nullptr, "out is NULL");
    auto h = std::make_unique<ckks_ctx>();
    ctx_init(h->c, log_n, q0_bits, scale_bits, n_scale, p_bits, n_special, device);
    *out = h.release();
  });
}

int ckks_context_destroy(ckks_ctx* ctx) {
  return guard([&] { delete ctx; });
}

int ckks_context_info(const ckks_ctx* ctx, uint64_t* moduli, double* delta, int* n_qp) {
  return guard([&] {
    need(ctx != nullptr, "ctx is NULL");
    const Ctx& c = ctx->c;
    if (moduli) memcpy(moduli, c.mod.data(), c.mod.size() * 8);
    if (delta) memcpy(delta, c.delta.data(), c.delta.size() * 8);
    if (n_qp) *n_qp = c.n_qp;
  });
}

int ckks_set_stream(ckks_ctx* ctx, void* stream) {
  return guard([&] {
    need(ctx != nullptr, "ctx is NULL");
    Ctx& c = ctx->c;
    CK_CUDA(cudaStreamSynchronize(c.stream));
    if (stream == nullptr) return;
    if (c.own_stream) CK_CUDA(cudaStreamDestroy(c.stream));
    c.own_stream = false;
    c.stream = static_cast<cudaStream_t>(stream);
  });
}

int ckks_set_fusion(ckks_ctx* ctx, int enabled) {
  return guard([&] {
    need(ctx != nullptr, "ctx is NULL");
    ctx->c.fused = enabled != 0;
  });
}

int ckks_synchronize(ckks_ctx* ctx) {
  return guard([&] {
    need(ctx != nullptr, "ctx is NULL");
    CK_CUDA(cudaStreamSynchronize(ctx->c.stream));
    ctx->c.check_waits();
  });
}

int ckks_selftest_wait(ckks_ctx* ctx, long long limit_cycles) {
  return guard([&] {
    need(ctx != nullptr, "ctx is NULL");
    need(limit_cycles >= 1 && limit_cycles <= (1ll << 32), "limit_cycles out of range");
    CK_CUDA(cudaStreamSynchronize(ctx->c.stream));
    ctx->c.check_waits();
    wait_selftest(ctx->c, limit_cycles);
    ctx->c.check_waits();
  });
}

int ckks_kernel_kind_count(void) { return K_KIND_COUNT; }

const char* ckks_kernel_kind_name(int kind) { return kernel_kind_name(kind); }

int ckks_launch_counts(const ckks_ctx* ctx, uint64_t* counts, int cap) {
  return guard([&] {
    need(ctx && counts, "NULL argument");
    for (int k = 0; k < K_KIND_COUNT && k < cap; k++) counts[k] = ctx->c.launches[k];
  });
}

int ckks_profile_enable(ckks_ctx* ctx, int on) {
  return guard([&] {
    need(ctx != nullptr, "ctx is NULL");
    ctx->c.prof = on != 0;
  });
}

int ckks_profile_collect(ckks_ctx* ctx, double* ms, double* bytes, uint64_t* launches, int cap) {
  return ckks_profile_collect2(ctx, ms, bytes, nullptr, launches, cap);
}

int ckks_profile_collect2(ckks_ctx* ctx, double* ms, double* bytes, double* modmuls,
                          uint64_t* launches, int cap) {
  return guard([&] {
    need(ctx != nullptr, "ctx is NULL");
    Ctx& c = ctx->c;
    CK_CUDA(cudaStreamSynchronize(c.stream));
    for (int k = 0; k < cap; k++) {
      if (ms) ms[k] = 0;
      if (bytes) bytes[k] = 0;
      if (modmuls) modmuls[k] = 0;
      if (launches) launches[k] = 0;
    }
    for (auto& r : c.prof_recs) {
      float t = 0;
      CK_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
      if (r.kind < cap) {
        if (ms) ms[r.kind] += t;
        if (bytes) bytes[r.kind] += r.bytes;
        if (modmuls) modmuls[r.kind] += r.ops;
        if (launches) launches[r.kind] += 1;
      }
      c.ev_pool.push_back(r.a);
      c.ev_pool.push_back(r.b);
    }
    c.prof_recs.clear();
    for (int k = 0; k < K_KIND_COUNT && k < cap; k++) {
      if (ms) ms[k] += c.prof_acc[k][0];
      if (bytes) bytes[k] += c.prof_acc[k][1];
      if (modmuls) modmuls[k] += c.prof_acc[k][2];
      if (launches) launches[k] += (uint64_t)c.prof_acc[k][3];
    }
    memset(c.prof_acc, 0, sizeof(c.prof_acc));
  });
}

int ckks_ntt(ckks_ctx* ctx, uint64_t* d_rows, size_t n_rows, int limbs, int inverse) {
  return guard([&] {
    need(ctx && d_rows, "NULL argument");
    Ctx& c = ctx->c;
    need(limbs >= 1 && limbs <= c.n_qp, "limbs out of range");
    if (inverse)
      ntt_inverse(c, d_rows, n_rows, c.iota(), limbs);
    else
      ntt_forward(c, d_rows, n_rows, c.iota(), limbs);
  });
}

int ckks_keygen(ckks_ctx* ctx, uint64_t seed, const int32_t* rot_steps, size_t n_steps,
                ckks_keys** out) {
  return guard([&] {
    need(ctx && out, "NULL argument");
    need(n_steps == 0 || rot_steps, "rot_steps is NULL");
    std::vector<int64_t> steps(rot_steps, rot_steps + n_steps);
    *out = keygen(ctx->c, seed, steps).release();
  });
}

int ckks_keys_compress(ckks_keys* keys) {
  return guard([&] {
    need(keys != nullptr, "NULL argument");
    keys_compress(*keys->ctx, *keys);
  });
}

int ckks_keys_bytes(const ckks_keys* keys, size_t* bytes) {
  return guard([&] {
    need(keys && bytes, "NULL argument");
    size_t b = keys->s.bytes + keys->relin.bytes;
    for (auto& kv : keys->galois) b += kv.second->bytes;
    *bytes = b;
  });
}

int ckks_keys_destroy(ckks_keys* keys) {
  return guard([&] { delete keys; });
}

int ckks_keys_export_secret(const ckks_keys* keys, uint64_t* host, size_t cap_words) {
  return guard([&] {
    need(keys && host, "NULL argument");
    need(cap_words * 8 >= keys->s.bytes, "buffer too small");
    Ctx& c = *keys->ctx;
    CK_CUDA(cudaMemcpyAsync(host, keys->s.p, keys->s.bytes, cudaMemcpyDeviceToHost, c.stream));
    CK_CUDA(cudaStreamSynchronize(c.stream));
  });
}

int ckks_keys_export_switch(const ckks_keys* keys, uint64_t galois, uint64_t* host,
                            size_t cap_words) {
  return guard([&] {
    need(keys && host, "NULL argument");
    Ctx& c = *keys->ctx;
    const size_t bytes = (size_t)c.beta_max * 2 * c.n_qp * c.N * 8;
    need(cap_words * 8 >= bytes, "buffer too small");
    DevBuf tmp;
    const uint64_t* w = switch_key_words(c, *keys, galois, tmp);
    CK_CUDA(cudaMemcpyAsync(host, w, bytes, cudaMemcpyDeviceToHost, c.stream));
    CK_CUDA(cudaStreamSynchronize(c.stream));
  });
}

uint64_t ckks_galois_element(const ckks_ctx* ctx, int32_t step) {
  return ctx ? ctx->c.galois(step) : 0;
}

int ckks_encrypt(ckks_ctx* ctx, const ckks_keys* keys, const double* values, size_t batch,
                 size_t n, int level, uint64_t seed, uint64_t first_index, ckks_ct** out) {
  return guard([&] {
    need(ctx && keys && out, "NULL argument");
    need(batch >= 1, "batch must be >= 1");
    need(n == 0 || values, "values is NULL");
    *out = encrypt(ctx->c, *keys, values, batch, n, level, seed, first_index).release();
  });
}

int ckks_decrypt(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* ct, double* out, size_t n) {
  return guard([&] {
    need(ctx && keys && ct && (out || n == 0), "NULL argument");
    decrypt(ctx->c, *keys, *ct, out, n);
  });
}

int ckks_ct_info(const ckks_ct* ct, size_t* batch, int* level, double* scale) {
  return guard([&] {
    need(ct != nullptr, "ct is NULL");
    if (batch) *batch = ct->B;
    if (level) *level = ct->level;
    if (scale) *scale = ct->scale;
  });
}

int ckks_ct_export(const ckks_ct* ct, uint64_t* host, size_t cap_words) {
  return guard([&] {
    need(ct && host, "NULL argument");
    need(cap_words >= ct->words(), "buffer too small");
    Ctx& c = *ct->ctx;
    CK_CUDA(cudaMemcpyAsync(host, ct->d.p, ct->d.bytes, cudaMemcpyDeviceToHost, c.stream));
    CK_CUDA(cudaStreamSynchronize(c.stream));
  });
}

int ckks_ct_import(ckks_ctx* ctx, const uint64_t* host, size_t batch, int level, double scale,
                   ckks_ct** out) {
  return guard([&] {
    need(ctx && host && out, "NULL argument");
    need(batch >= 1, "batch must be >= 1");
    Ctx& c = ctx->c;
    Ct r = ct_alloc(c, batch, level, scale);
    CK_CUDA(cudaMemcpyAsync(r->d.p, host, r->d.bytes, cudaMemcpyHostToDevice, c.stream));
    CK_CUDA(cudaStreamSynchronize(c.stream));
    *out = r.release();
  });
}

int ckks_ct_import_async(ckks_ctx* ctx, const uint64_t* host, size_t batch, int level,
                         double scale, void* copy_stream, ckks_ct** out) {
  return guard([&] {
    need(ctx && host && out && copy_stream, "NULL argument");
    need(batch >= 1, "batch must be >= 1");
    need(level >= 0 && level <= ctx->c.L, "level out of range");
    Ctx& c = ctx->c;
    cudaStream_t cs = static_cast<cudaStream_t>(copy_stream);
    auto r = std::make_unique<ckks_ct>();
    r->ctx = &c;
    r->B = batch;
    r->level = level;
    r->scale = scale;
    // allocated in the copy stream's order (freed later in the library's)
    const size_t bytes = batch * 2 * (size_t)(level + 1) * c.N * 8;
    CK_CUDA(cudaMallocAsync(&r->d.p, bytes, cs));
    r->d.ctx = &c;
    r->d.bytes = bytes;
    CK_CUDA(cudaMemcpyAsync(r->d.p, host, bytes, cudaMemcpyHostToDevice, cs));
    cudaEvent_t e;
    CK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CK_CUDA(cudaEventRecord(e, cs));
    CK_CUDA(cudaStreamWaitEvent(c.stream, e, 0));
    CK_CUDA(cudaEventDestroy(e));
    *out = r.release();
  });
}

int ckks_ct_slice(ckks_ctx* ctx, const ckks_ct* ct, size_t first, size_t count, ckks_ct** out) {
  return guard([&] {
    need(ctx && ct && out, "NULL argument");
    need(count >= 1 && first + count <= ct->B, "slice out of range");
    Ctx& c = ctx->c;
    Ct r = ct_alloc(c, count, ct->level, ct->scale);
    const size_t per = ct->words() / ct->B;
    CK_CUDA(cudaMemcpyAsync(r->d.p, ct->d.u64() + first * per, r->d.bytes,
                            cudaMemcpyDeviceToDevice, c.stream));
    *out = r.release();
  });
}

int ckks_ct_destroy(ckks_ct* ct) {
  return guard([&] { delete ct; });
}

#define BINARY(name, body)                                                       \
  int name(ckks_ctx* ctx, const ckks_ct* a, const ckks_ct* b, ckks_ct** out) {  \
    return guard([&] {                                                           \
      need(ctx && a && b && out, "NULL argument");                               \
      *out = (body).release();                                                   \
    });                                                                          \
  }

BINARY(ckks_add, op_add(ctx->c, *a, *b, false))
BINARY(ckks_sub, op_add(ctx->c, *a, *b, true))

int ckks_mul_relin(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* a, const ckks_ct* b,
                   ckks_ct** out) {
  return guard([&] {
    need(ctx && keys && a && b && out, "NULL argument");
    need(a->B == b->B, "batch sizes differ");
    if (a->level != b->level) throw Error(CKKS_ERR_LEVEL, "levels differ");
    *out = op_mul_relin(ctx->c, *keys, *a, *b).release();
  });
}

int ckks_rescale(ckks_ctx* ctx, const ckks_ct* in, ckks_ct** out) {
  return guard([&] {
    need(ctx && in && out, "NULL argument");
    *out = op_rescale(ctx->c, *in).release();
  });
}

int ckks_mul(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* a, const ckks_ct* b,
             ckks_ct** out) {
  return guard([&] {
    need(ctx && keys && a && b && out, "NULL argument");
    need(a->B == b->B, "batch sizes differ");
    *out = op_mul(ctx->c, *keys, *a, *b).release();
  });
}

int ckks_mul_plain(ckks_ctx* ctx, const ckks_ct* a, const double* v, size_t n, ckks_ct** out) {
  return guard([&] {
    need(ctx && a && out && (v || n == 0), "NULL argument");
    Ctx& c = ctx->c;
    if (a->level < 1) throw Error(CKKS_ERR_LEVEL, "level exhausted");
    const double S = plain_scale(c, a->scale, a->level);
    DevBuf pt = encode_vec(c, v, n, a->level, S);
    *out = op_mul_pt(c, *a, pt.u64(), S).release();
  });
}

int ckks_add_plain(ckks_ctx* ctx, const ckks_ct* a, const double* v, size_t n, ckks_ct** out) {
  return guard([&] {
    need(ctx && a && out && (v || n == 0), "NULL argument");
    Ctx& c = ctx->c;
    DevBuf pt = encode_vec(c, v, n, a->level, a->scale);
    *out = op_add_pt(c, *a, pt.u64()).release();
  });
}

int ckks_mul_const(ckks_ctx* ctx, const ckks_ct* a, double v, ckks_ct** out) {
  return guard([&] {
    need(ctx && a && out, "NULL argument");
    if (a->level < 1) throw Error(CKKS_ERR_LEVEL, "level exhausted");
    *out = op_mul_const(ctx->c, *a, v).release();
  });
}

int ckks_add_const(ckks_ctx* ctx, const ckks_ct* a, double v, ckks_ct** out) {
  return guard([&] {
    need(ctx && a && out, "NULL argument");
    *out = op_add_const(ctx->c, *a, v).release();
  });
}

int ckks_level_down(ckks_ctx* ctx, const ckks_ct* a, int level, ckks_ct** out) {
  return guard([&] {
    need(ctx && a && out, "NULL argument");
    if (level < 0 || level > a->level) throw Error(CKKS_ERR_LEVEL, "level out of range");
    *out = op_level_down(ctx->c, *a, level).release();
  });
}

int ckks_rotate(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* in, int32_t step,
                ckks_ct** out) {
  return guard([&] {
    need(ctx && keys && in && out, "NULL argument");
    *out = op_rotate(ctx->c, *keys, *in, step).release();
  });
}

int ckks_rotate_hoisted(ckks_ctx* ctx, const ckks_keys* keys, const ckks_ct* in,
                        const int32_t* steps, size_t n_steps, ckks_ct** outs) {
  return guard([&] {
    need(ctx && keys && in && outs && (steps || n_steps == 0), "NULL argument");
    std::vector<int64_t> s(steps, steps + n_steps);
    auto r = op_rotate_many(ctx->c, *keys, *in, s);
    for (size_t i = 0; i < n_steps; i++) outs[i] = r[i].release();
  });
}

}  // extern "C"
