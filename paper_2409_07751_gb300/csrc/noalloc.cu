// Allocation-free rescale for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the
// point where they rescale: code running while a CUDA stream is being
// captured into a graph, runtimes that hand out a fixed device-memory budget
// up front, or real-time loops that forbid allocator calls. For them this
// file keeps the rescale's working memory (the copied top limb and the
// spread correction term) in one file-scope device array of fixed size
// instead of asking an allocator for it. The caller still passes the input
// and output ciphertext memory.
//
// The array is sized for 8 Mi words (64 MiB); every GPU that loads this
// library holds it until the process exits. Its address is looked up once
// per device on the first call (with that device current), so the first call
// on each device should happen before any stream capture. All calls share
// the array: two calls that overlap on the GPU (different streams, or
// different host threads) race on it and must be serialized by the caller.
// Both scratch regions are fully written before they are read, so nothing
// in the array needs clearing between calls. The calling thread's current
// device is the same after the call as before it.
#include <mutex>

#include "ops.h"

using namespace ck;

namespace {

constexpr size_t NOALLOC_SCRATCH_WORDS = (size_t)8 << 20;
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) uint64_t g_noalloc_scratch[NOALLOC_SCRATCH_WORDS];

std::mutex g_mu;
uint64_t* g_scratch_addr[MAX_DEVICES] = {};

// Device address of the scratch array on `device` (host code must not use
// the array's name as a device pointer).
uint64_t* scratch_on(int device) {
  if (device < 0 || device >= MAX_DEVICES) throw Error(CKKS_ERR_UNSUPPORTED, "device ordinal >= 64");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;  // `device` is current (set by the caller below)
    CK_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_addr[device] = static_cast<uint64_t*>(p);
  }
  return g_scratch_addr[device];
}

// Restores the calling thread's current device when the call returns.
struct CurrentDeviceGuard {
  int prev = -1;
  CurrentDeviceGuard() {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  }
  ~CurrentDeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

bool overlaps(const uint64_t* a, size_t na, const uint64_t* b, size_t nb) {
  const uintptr_t a0 = (uintptr_t)a, a1 = a0 + na * 8, b0 = (uintptr_t)b, b1 = b0 + nb * 8;
  return a0 < b1 && b0 < a1;
}

}  // namespace

extern "C" int ckks_rescale_noalloc(ckks_ctx* ctx, const uint64_t* d_in, size_t batch, int level,
                                    uint64_t* d_out) {
  try {
    if (!ctx || !d_in || !d_out || batch == 0) return CKKS_ERR_INVALID_ARG;
    Ctx& c = ctx->c;
    if (level < 1 || level > c.L) return CKKS_ERR_LEVEL;
    // 2 batch N (level + 1) scratch words, bounded before it is formed so
    // that no product can wrap around
    const size_t per_ct = 2 * c.N * (size_t)(1 + level);
    if (batch > NOALLOC_SCRATCH_WORDS / per_ct) return CKKS_ERR_INVALID_ARG;
    const size_t polys = 2 * batch;
    // the output limbs are strided differently from the input's: in place
    // (or any overlap) would read words already overwritten
    if (overlaps(d_in, batch * per_ct, d_out, polys * c.N * (size_t)level))
      return CKKS_ERR_INVALID_ARG;
    CurrentDeviceGuard restore;
    CK_CUDA(cudaSetDevice(c.device));
    uint64_t* last = scratch_on(c.device);
    uint64_t* R = last + polys * c.N;
    CK_CUDA(cudaMemcpy2DAsync(last, c.N * 8, d_in + (size_t)level * c.N,
                              (size_t)(level + 1) * c.N * 8, c.N * 8, polys,
                              cudaMemcpyDeviceToDevice, c.stream));
    ntt_inverse(c, last, polys, c.iota() + level, 1);
    k_rescale_spread(c, last, R, polys, level);
    ntt_forward(c, R, polys * level, c.iota(), level);
    k_rescale_finish(c, d_in, R, d_out, polys, level, c.d_rs_inv.u64() + (size_t)level * (c.L + 1),
                     c.d_rs_invs.u64() + (size_t)level * (c.L + 1));
    return CKKS_OK;
  } catch (...) {
    return api_error();
  }
}
